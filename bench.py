"""Benchmark: FDA matvec/s and GMRES solve time for the rigid-sphere Burton-Miller problem at kD = 200.

Workload (default): sphere of radius 0.5 (D = 1) at k = 200, icosphere frequency 97: 188,180 curved
quadratic triangles, N = 1,129,080 DOF (the paper's kD ~ 200 sphere with h ~ lambda/5), FDA eps = 1e-4,
<= 64 points per leaf, seeded complex Gaussian density, plane wave along +z for the solves.

A step is one FDA matrix-vector product of the whole operator (near field + S2M + M2M + M2L + L2L + L2T)
on one batch of nrhs densities, inputs resident in HBM. `value` is matvec/s of the mixed-precision
form (FP32 near field and translations); the plain FP64 form is reported beside it, and so are the GMRES
solve times to a 1e-5 relative residual (plain FP64 GMRES vs FP64 iterative refinement around the FP32
operator). The operator data (GBs) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Multi-GPU: replicas only (every rank runs the same workload, no collective on the data path);
value = all ranks' matvecs / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1311_5202_gb300 import inputs  # noqa: E402

METRIC = "FDA matvec/s and GMRES solve s at kD=200: mixed+learned vs plain FP64, same GB300"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def mie_surface(xs, k, a, chunk=100000):
    """Total field on a rigid sphere of radius a for u_inc = exp(i k z) (the Mie series of Sec. 5.3 with the
    first-kind Hankel function of G = e^{ikr}/(4 pi r)): by the Wronskian of j_n and y_n,
    u(theta) = (i/z^2) sum_n (2n+1) i^n P_n(cos theta)/h_n'(z), z = ka. Evaluated with scipy's spherical
    Bessel functions; it only reports the accuracy of a solve."""
    from scipy.special import spherical_jn, spherical_yn
    z = k * a
    nmax = int(z + 10 * z ** (1.0 / 3.0) + 10)
    n = np.arange(nmax + 1)
    dh = spherical_jn(n, z, derivative=True) + 1j * spherical_yn(n, z, derivative=True)
    coef = (2 * n + 1) * (1j ** n) / dh
    c = xs[:, 2] / np.linalg.norm(xs, axis=1)
    out = np.empty(len(c), dtype=np.complex128)
    for i0 in range(0, len(c), chunk):
        x = c[i0:i0 + chunk]
        p0, p1 = np.ones_like(x), x.copy()
        acc = coef[0] * p0 + coef[1] * p1
        for m in range(1, nmax):
            p0, p1 = p1, ((2 * m + 1) * x * p1 - m * p0) / (m + 1)
            acc += coef[m + 1] * p1
        out[i0:i0 + chunk] = acc
    return (1j / z ** 2) * out


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, gpu_index=0):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return out
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(gpu_index)]
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def max_over_ranks(value, dist, device):
    """Largest value over the ranks of the default process group (timings are reported max-over-ranks)."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size, nrhs, ms_per_step):
    """Whole-job right-hand-side matvecs per second: every replica does nrhs per step."""
    return world_size * nrhs * 1000.0 / ms_per_step


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(mesh, k, x, rows_n, seed=7):
    """The FP64 oracle (dense Nystrom rows, O(N) each) on a bounded sample of rows, all host cores."""
    from oracle import oracle as O
    N = mesh.n_dof
    rows = inputs.sample_rows(N, rows_n, seed)
    t0 = time.perf_counter()
    O.matvec_rows(mesh.nodes, mesh.elems, k, x, rows)
    dt = time.perf_counter() - t0
    per_matvec = dt * N / len(rows)
    return {"value": 1.0 / per_matvec, "unit": "matvec/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{len(rows)} of {N} rows of the dense FP64 oracle matvec (O(N) each, locally corrected), "
                      f"{dt:.2f} s wall, extrapolated x N/rows"}


def workload_config(args, spec, mesh, ws):
    """The `config` object of both arms: the workload by name and size."""
    k = spec["k"]
    return {"workload": args.workload, "N": mesh.n_dof, "k": k, "kD": k * float(np.ptp(mesh.nodes, axis=0).max()),
            "eps": args.eps or spec["eps"], "leaf_max": spec["leaf"], "nrhs": args.nrhs,
            "parallelism": f"replicas{ws}", "l2": "operators and vectors (GBs) larger than L2; no flush"}


def run_reference(args):
    """Reference arm: the oracle as it stands, on this machine's host cores, same workload, metric and unit."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    spec = inputs.WORKLOADS[args.workload]
    mesh = inputs.make_mesh(spec)
    k = spec["k"]
    x = inputs.complex_gaussian(mesh.n_dof, 20131120)
    rows_per_step = args.ref_rows
    from oracle import oracle as O
    for _ in range(args.warmup):
        O.matvec_rows(mesh.nodes, mesh.elems, k, x, inputs.sample_rows(mesh.n_dof, max(4, rows_per_step // 4), 1))
    times = []
    for s in range(args.steps):
        rows = inputs.sample_rows(mesh.n_dof, rows_per_step, 100 + s)
        t0 = time.perf_counter()
        O.matvec_rows(mesh.nodes, mesh.elems, k, x, rows)
        times.append(time.perf_counter() - t0)
    per_matvec = float(np.mean(times)) * mesh.n_dof / rows_per_step
    value = 1.0 / per_matvec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_matvec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": workload_config(args, spec, mesh, ws),
            "cpu_baseline": {"value": value, "unit": "matvec/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{rows_per_step} sampled rows per step of the dense FP64 oracle matvec, "
                                       f"extrapolated x N/rows"},
            "e2e": {"value": value, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(S2, args, N, dev, stream, single_mixed, fdbem, torch):
    """Many incident directions at once on the alpha = -i/k plan: autotuned, graph-captured batched matvec
    (right-hand-side matvecs per second) and a lockstep block solve of the plane waves to 1e-5."""
    B = args.batch
    tune = None if args.no_tune else fdbem.fda_autotune(S2.plan, B)
    X = inputs.complex_gaussian(N, 20131121, nrhs=B).astype(np.complex64)
    xb = torch.from_numpy(X).to(dev).contiguous()
    yb = torch.empty_like(xb)
    reps = max(2, args.steps // 2)

    def clock(fn, n):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    # single-pass TF32 translations (on a plan with 3xTF32 images, their leading part)
    ms_direct = clock(lambda: fdbem.fda_matvec_ex(S2.plan, fdbem.FDA_PREC_TF32, xb, yb, stream), reps)
    g = fdbem.fda_matvec_graph_create(S2.plan, fdbem.FDA_PREC_TF32, xb, yb, stream)
    try:
        nodes = fdbem.fda_graph_nodes(g)
        ms_graph = clock(lambda: fdbem.fda_graph_launch(g, stream), reps)
    finally:
        fdbem.fda_graph_destroy(g)
    ph = fdbem.fda_matvec_phases(S2.plan, fdbem.FDA_PREC_TF32, xb, yb, stream)
    dirs = inputs.fibonacci_directions(B)
    b = torch.empty((B, N), dtype=torch.complex128, device=dev)
    fdbem.bm_rhs_plane_wave(S2.prob, dirs, b, stream)
    xs = torch.zeros_like(b)
    t1 = time.perf_counter()
    st = fdbem.bm_gmres_solve(S2.plan, b, xs, tol=1e-5, restart=60, max_iter=2000, refine=True, inner_tol=1e-3,
                              stream=stream, raise_on_error=False)
    torch.cuda.synchronize()
    st["wall_s"] = time.perf_counter() - t1
    st["per_direction_s"] = st["wall_s"] / B
    out = {"nrhs": B, "directions": "Fibonacci sphere", "rhs_matvec_per_s": B * 1000.0 / ms_direct,
           "rhs_matvec_per_s_graph": B * 1000.0 / ms_graph, "ms_per_batched_matvec": ms_direct,
           "ms_per_batched_matvec_graph": ms_graph, "graph_nodes": nodes, "phase_ms": ph, "autotune": tune,
           "block_solve_mixed": st}
    if single_mixed:
        out["speedup_per_direction_vs_single_mixed_solve"] = single_mixed["wall_s"] / st["per_direction_s"]
    if args.solve_m2l_tensor == 3:
        # the same block solve with the 3xTF32 product as the outer residual; it stops at 0.9e-5, since over many
        # directions the worst FP64 residual sits further from the 3xTF32 one (reported beside)
        xs3 = torch.zeros_like(b)
        t2 = time.perf_counter()
        st3 = fdbem.bm_gmres_solve(S2.plan, b, xs3, tol=0.9e-5, restart=60, max_iter=2000, refine=True,
                                   inner_tol=1e-3, stream=stream, raise_on_error=False, refine_residual=1)
        torch.cuda.synchronize()
        st3["wall_s"] = time.perf_counter() - t2
        st3["per_direction_s"] = st3["wall_s"] / B
        r = torch.empty_like(b)
        fdbem.fda_matvec_ex(S2.plan, fdbem.FDA_PREC_FP64, xs3, r, stream)
        torch.cuda.synchronize()
        st3["rel_residual_fp64_worst"] = float((torch.linalg.norm(b - r, dim=1) / torch.linalg.norm(b, dim=1)).max())
        out["block_solve_mixed_3xtf32_residual"] = st3
    return out


def direct_particle_rows(x, n, k, q, rows, alpha, chunk=1 << 16):
    """p_i = sum_{j != i} [G + alpha dG/dn_y](x_i, y_j) q_j for the sampled targets i (Sec. 5.1, Eq. sum),
    plainly in numpy FP64, with G = e^{ikR}/(4 pi R) and dG/dn_y = G (1/R - ik) (r.n_y)/R, r = x_i - y_j; it
    only reports the accuracy of the FDA product."""
    out = np.zeros(len(rows), dtype=np.complex128)
    for t, i in enumerate(rows):
        acc = 0j
        for j0 in range(0, len(x), chunk):
            y, ny, qj = x[j0:j0 + chunk], n[j0:j0 + chunk], q[j0:j0 + chunk]
            r = x[i] - y
            R = np.sqrt(np.sum(r * r, axis=1))
            self_term = R == 0  # the j = i term is excluded
            R[self_term] = 1.0
            G = np.exp(1j * k * R) / (4 * np.pi * R)
            dG = G * (1.0 / R - 1j * k) * np.sum(r * ny, axis=1) / R
            acc += np.sum(np.where(self_term, 0.0, (G + alpha * dG) * qj))
        out[t] = acc
    return out


def table1_case(N, k, eps, fdbem, torch, dev, stream, tune=True, reps=3):
    """One particle summation of the paper's Table 1 (Sec. 5.1, Eq. sum): unit sphere, ~20 points per
    wavelength, zero-mean random densities; the FDA product in FP64, in the mixed form with TF32 translations
    and in the mixed form with 3xTF32 translations (FP32 level), its phases, and eps_a over 200 random targets
    against the direct sum (the paper's error measure)."""
    x, n = inputs.sphere_points(N, 1.0)
    q = inputs.complex_gaussian(N, 20131120)
    rows = inputs.sample_rows(N, 200, 5)
    t1 = time.perf_counter()
    po = direct_particle_rows(x, n, k, q, rows, 1j / k)
    out = {"N": N, "k": k, "eps": eps, "direct_200_rows_s": time.perf_counter() - t1}
    for m2lt, forms in ((1, ((fdbem.FDA_PREC_FP64, "fp64"), (fdbem.FDA_PREC_FP32, "mixed"))),
                        (3, ((fdbem.FDA_PREC_FP32, "mixed_3xtf32"),))):
        t0 = time.perf_counter()
        P = fdbem.ParticleSum(x, n, k, eps=eps, leaf_max=64, precision=fdbem.FDA_PREC_FP32, m2l_tensor=m2lt)
        setup = time.perf_counter() - t0
        try:
            if tune:
                fdbem.fda_autotune(P.plan, 1)
            info = P.info()
            if m2lt == 1:
                out.update({"setup_s": setup, "device_gb": info["device_bytes"] / 1e9})
            else:
                out["device_gb_3xtf32"] = info["device_bytes"] / 1e9
            qd = torch.from_numpy(q).to(dev)
            pd = torch.empty_like(qd)
            for prec, name in forms:
                fdbem.fda_matvec_ex(P.plan, prec, qd, pd, stream)
                torch.cuda.synchronize()
                pa = pd.cpu().numpy()[rows]
                err = float(np.sqrt(np.sum(np.abs(pa - po) ** 2) / np.sum(np.abs(po) ** 2)))
                phs = [fdbem.fda_matvec_phases(P.plan, prec, qd, pd, stream) for _ in range(reps)]
                ph = {key: float(np.median([p_[key] for p_ in phs])) for key in phs[0]}
                out[name] = {"eps_a": err, "ms": sum(ph.values()), "m2l_ms": ph["m2l"],
                             "up_ms": ph["s2m"] + ph["m2m"], "down_ms": ph["l2l"] + ph["l2t"], "near_ms": ph["near"]}
        finally:
            P.close()
    return out


def run_table1(args):
    import torch
    from paper_1311_5202_gb300 import fdbem
    ws, rank, local = dist_setup()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rows = []
    for N, k in inputs.TABLE1[: args.table1_max]:
        for eps in args.table1_eps:
            rows.append(table1_case(N, k, eps, fdbem, torch, dev, stream, tune=not args.no_tune))
            print(json.dumps({"table1_row": rows[-1]}), file=sys.stderr, flush=True)
    print(json.dumps({"table1": rows, "unit_ms": "per product on one GB300",
                      "paper": "Table 1, one Xeon 5450 core, T_M2L and T_up in seconds"}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="sphere_kd200", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--ref-rows", type=int, default=48)
    ap.add_argument("--cpu-rows", type=int, default=192)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-alt", action="store_true", help="skip the alpha = -i/k solves")
    ap.add_argument("--no-plus-solve", action="store_true",
                    help="skip the solve with the coupling alpha = +i/k (its ring spectrum needs thousands of "
                         "iterations on elongated bodies)")
    ap.add_argument("--full-solve", action="store_true", help="also the plain FP64 solve at alpha = i/k (long)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip training/using the learned preconditioner")
    ap.add_argument("--eps", type=float, default=None)
    ap.add_argument("--m2l-tensor", type=int, default=1, choices=[0, 1, 2],
                    help="M2L of the FP32 form: 0 FP32 FMA, 1 TF32 tensor cores, 2 3xTF32 tensor cores")
    ap.add_argument("--batch", type=int, default=16,
                    help="directions of the batched section (autotuned, graph-captured matvec and block solve); "
                         "0 skips it")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner")
    ap.add_argument("--m2l-variant", type=int, default=None,
                    help="pin one M2L kernel variant for every level and stage instead of autotuning "
                         "(fda_m2l_force; used to profile one kernel)")
    ap.add_argument("--overlap", type=int, default=None, choices=[0, 1, 2, 3],
                    help="force the FP32 product schedule instead of the autotuner's (0 serial; 1, 2, 3 far field "
                         "on a second stream beside the near field at two, one or three CTAs per SM; "
                         "fda_overlap_force)")
    ap.add_argument("--near-evict", type=int, default=None, choices=[0, 1],
                    help="force the L2 policy of the near-field matrix copies (1 evict-first) instead of the "
                         "autotuner's")
    ap.add_argument("--near-form", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="near-field form of the product plan before autotuning (fda_config_t.near_form; with "
                         "--no-tune it stays: 4 = the tensor-core form for batches)")
    ap.add_argument("--far-levels", type=int, default=None, choices=[0, 1],
                    help="force the M2L levels onto concurrent streams (1) or in sequence (0) instead of the "
                         "autotuner's choice")
    ap.add_argument("--solve-m2l-tensor", type=int, default=3, choices=[1, 3],
                    help="tensor-core images of the alpha = -i/k solve plan: 3 (3xTF32; adds the solves with the "
                         "3xTF32 outer residual) or 1 (TF32)")
    ap.add_argument("--table1", action="store_true",
                    help="run only the particle summations of the paper's Table 1 and print their JSON line")
    ap.add_argument("--table1-max", type=int, default=3, help="number of Table 1 sizes (4 adds N = 4.7M)")
    ap.add_argument("--table1-eps", type=float, nargs="+", default=[1e-4, 1e-6])
    ap.add_argument("--no-table1-sample", action="store_true", help="skip the Table 1 case in the default run")
    ap.add_argument("--near-split", type=int, default=0, choices=[0, 1, 2],
                    help="near-field correction schedule of the plan before the autotuner (with --no-tune: kept)")
    ap.add_argument("--clocks-dir", default=None,
                    help="where the nvidia-smi clock samples of the timed region are kept (default: temp dir)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.table1:
        return run_table1(args)

    import torch
    from paper_1311_5202_gb300 import fdbem

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    dev = torch.device("cuda", local)
    spec = inputs.WORKLOADS[args.workload]
    eps = args.eps or spec["eps"]
    mesh = inputs.make_mesh(spec)
    k = spec["k"]
    N = mesh.n_dof
    nrhs = args.nrhs
    t0 = time.perf_counter()
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=eps, leaf_max=spec["leaf"], precision=fdbem.FDA_PREC_FP32,
                     lowrank=1, nrhs_max=nrhs, m2l_tensor=args.m2l_tensor, near_split=args.near_split,
                     near_form=args.near_form)
    setup_s = time.perf_counter() - t0
    tune_main = None if (args.no_tune or args.m2l_variant is not None) else fdbem.fda_autotune(S.plan, nrhs)
    if args.m2l_variant is not None:
        fdbem.fda_m2l_force(S.plan, args.m2l_variant)
    overlap = args.overlap if args.overlap is not None else (tune_main["overlap"] if tune_main else 0)
    evict = args.near_evict if args.near_evict is not None else (tune_main["near_evict_first"] if tune_main else 0)
    farp = args.far_levels if args.far_levels is not None else (tune_main["far_levels_concurrent"] if tune_main
                                                                 else 0)
    if args.overlap is not None or args.near_evict is not None or args.far_levels is not None:
        fdbem.fda_overlap_force(S.plan, overlap, evict, farp)
    info = S.info()
    X = inputs.complex_gaussian(N, 20131120, nrhs=nrhs if nrhs > 1 else None)
    xd = torch.from_numpy(X).to(dev).contiguous()
    yd = torch.empty_like(xd)
    stream = torch.cuda.current_stream()

    def timed(prec, steps, warm):
        for _ in range(warm):
            fdbem.fda_matvec_ex(S.plan, prec, xd, yd, stream)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # an NVTX range names the timed products, so that a profiler can keep to them (ncu --nvtx-include)
        torch.cuda.nvtx.range_push("mixed_matvec" if prec == fdbem.FDA_PREC_FP32 else "fp64_matvec")
        e0.record(stream)
        for _ in range(steps):
            fdbem.fda_matvec_ex(S.plan, prec, xd, yd, stream)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if pg:
            ms = max_over_ranks(ms, pg, dev)
        return ms

    clocks = Clocks(os.path.join(args.clocks_dir or tempfile.gettempdir(), f"bench_clocks_r{rank}.csv"))
    with clocks:
        ms32 = timed(fdbem.FDA_PREC_FP32, args.steps, args.warmup)
        launches = int(S.info()["launches_per_matvec"])
    steps64 = max(3, args.steps // 3) if nrhs == 1 else 1
    ms64 = timed(fdbem.FDA_PREC_FP64, steps64, 1 if nrhs == 1 else 0)
    # phase breakdown (device time per phase, one launch each)
    ph32 = fdbem.fda_matvec_phases(S.plan, fdbem.FDA_PREC_FP32, xd, yd, stream)
    ph64 = fdbem.fda_matvec_phases(S.plan, fdbem.FDA_PREC_FP64, xd, yd, stream)
    # end to end through the C ABI with host buffers: H2D of x, matvec, D2H of y per step
    xh = torch.from_numpy(X).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        xd.copy_(xh, non_blocking=True)
        fdbem.fda_matvec_ex(S.plan, fdbem.FDA_PREC_FP32, xd, yd, stream)
        yh.copy_(yd, non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        fdbem.fda_matvec_ex(S.plan, fdbem.FDA_PREC_FP32, xd, yd, stream)
        yh.copy_(yd, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    if pg:
        e2e_ms = max_over_ranks(e2e_ms, pg, dev)
    # the Mie series on the Nystrom points (sphere workloads): accuracy of every plane-wave solve
    mie_ref = None
    if spec["kind"] == "sphere" and not args.no_solve:
        xg = torch.empty(N * 3, dtype=torch.float64, device=dev)
        fdbem.bm_problem_geometry(S.prob, xg, torch.empty_like(xg), torch.empty(N, dtype=torch.float64, device=dev))
        mie_ref = mie_surface(xg.cpu().numpy().reshape(N, 3), k, spec.get("radius", 0.5))

    def mie_err(xs):
        if mie_ref is None:
            return None
        return float(np.linalg.norm(xs.cpu().numpy() - mie_ref) / np.linalg.norm(mie_ref))

    # solves to 1e-5: plain FP64 GMRES vs FP64 iterative refinement around the FP32 operator
    def fp64_residual(Sx, b, xs):
        # relative residual of a solution against the FP64 operator (outside the timed solve)
        r = torch.empty_like(b)
        fdbem.fda_matvec_ex(Sx.plan, fdbem.FDA_PREC_FP64, xs, r, stream)
        torch.cuda.synchronize()
        return float(torch.linalg.norm(b - r) / torch.linalg.norm(b))

    def solves(Sx, kinds, restart, max_iter, tol=1e-5):
        out = {}
        b = torch.empty(N, dtype=torch.complex128, device=dev)
        fdbem.bm_rhs_plane_wave(Sx.prob, [0.0, 0.0, 1.0], b, stream)
        for name, kw in kinds:
            xs = torch.zeros_like(b)
            # the 3xTF32 outer residual differs from the FP64 one by a few 1e-7 (relative): these solves stop at
            # 0.95 tol, so that the FP64 residual of the result (reported beside) stays within tol; with
            # refine_residual = 2 the library confirms with the FP64 operator itself
            t_solve = 0.95 * tol if kw.get("refine_residual") == 1 else tol
            t1 = time.perf_counter()
            st = fdbem.bm_gmres_solve(Sx.plan, b, xs, tol=t_solve, restart=restart, max_iter=max_iter,
                                      stream=stream, raise_on_error=False, **kw)
            torch.cuda.synchronize()
            st["wall_s"] = time.perf_counter() - t1
            st["tol"] = t_solve
            st["mie_rel_l2"] = mie_err(xs)
            if kw.get("refine_residual"):
                st["rel_residual_fp64"] = fp64_residual(Sx, b, xs)
            out[name] = st
        return out

    solve = {}
    solve_alt = {}
    batched = None
    if not args.no_solve and not args.no_plus_solve:
        # coupling alpha = i/k as stated: its sphere spectrum rings the origin, so a large Krylov space
        kinds = [("mixed", dict(refine=True, inner_tol=1e-3))]
        if args.full_solve:
            kinds.insert(0, ("fp64", dict(refine=False)))
        solve = solves(S, kinds, 400, 4000)
        if args.full_solve:
            # the paper's GMRES tolerance of its kD = 314 sphere (Sec. 5.3: 14 iterations to 1e-3)
            solve["mixed_tol_1e-3"] = solves(S, [("mixed", dict(refine=True, inner_tol=1e-3))], 400, 4000,
                                             tol=1e-3)["mixed"]
    S.close()
    puls = None
    if not args.no_solve and not args.no_alt and spec["kind"] == "sphere":
        # radiation data of the pulsating sphere (Sec. 5.2): b = (Sbar + alpha Mbar - alpha/2) 1, operator B of
        # its own FP64 plan (freed before the solve plan is built)
        t5 = time.perf_counter()
        SB = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=eps, leaf_max=spec["leaf"], precision=fdbem.FDA_PREC_FP64,
                          lowrank=1, nrhs_max=1, alpha=-1j / k, op=1)
        b_puls = torch.empty(N, dtype=torch.complex128, device=dev)
        SB.matvec(torch.ones(N, dtype=torch.complex128, device=dev), b_puls, stream)
        torch.cuda.synchronize()
        SB.close()
        puls = {"setup_rhs_s": time.perf_counter() - t5}
    if not args.no_solve and not args.no_alt:
        # coupling alpha = -i/k: clustered spectrum, the iteration counts the paper reports
        t2 = time.perf_counter()
        # 3xTF32 images (m2l_tensor = 3): single-pass TF32 products for the inner solves, and the 3xTF32 FP32
        # product as the refinement's outer residual in the *_3xtf32_residual solves
        S2 = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=eps, leaf_max=spec["leaf"], precision=fdbem.FDA_PREC_FP32,
                          lowrank=1, nrhs_max=max(1, args.batch), alpha=-1j / k, m2l_tensor=args.solve_m2l_tensor)
        if not args.no_tune:
            fdbem.fda_autotune(S2.plan, 1)
        setup2 = time.perf_counter() - t2
        kinds = [("fp64", dict(refine=False)), ("mixed", dict(refine=True, inner_tol=1e-3))]
        if args.solve_m2l_tensor == 3:
            kinds.append(("mixed_3xtf32_residual", dict(refine=True, inner_tol=1e-3, refine_residual=1)))
            # the same, certified at the end with the FP64 operator (no margin needed)
            kinds.append(("mixed_3xtf32_residual_fp64_check", dict(refine=True, inner_tol=1e-3, refine_residual=2)))
        solve_alt = solves(S2, kinds, 100, 2000)
        solve_alt["mixed_tol_1e-3"] = solves(S2, [("mixed", dict(refine=True, inner_tol=1e-3))], 100, 2000,
                                             tol=1e-3)["mixed"]
        if args.solve_m2l_tensor == 3:
            solve_alt["mixed_3xtf32_residual_tol_1e-3"] = solves(
                S2, [("m", dict(refine=True, inner_tol=1e-3, refine_residual=1))], 100, 2000, tol=1e-3)["m"]
        solve_alt["setup_s"] = setup2
        if not args.no_learned:
            # learned leaf-block preconditioner: trained on seeded random ellipsoids (kD 20-40, 12k DOF each)
            # from the method's own GMRES solves, then flexible GMRES inside the mixed solve
            from paper_1311_5202_gb300 import precond as PCm
            t3 = time.perf_counter()
            train = [(inputs.ellipsoid(10, ax), kk) for ax, kk in
                     inputs.random_ellipsoid_params(3, seed=1, kd_range=(20.0, 40.0))]
            net, tinfo = PCm.build_trained(train, alpha_sign=-1, hidden=32, epochs=20, dirs_per_mesh=6)
            train_s = time.perf_counter() - t3
            pc = fdbem.bm_precond_create(S2.plan)
            b = torch.empty(N, dtype=torch.complex128, device=dev)
            fdbem.bm_rhs_plane_wave(S2.prob, [0.0, 0.0, 1.0], b, stream)
            xs = torch.zeros_like(b)
            t4 = time.perf_counter()
            st = fdbem.bm_fgmres_solve(S2.plan, pc, net, b, xs, tol=1e-5, restart=100, max_iter=2000, refine=True,
                                       inner_tol=1e-3, stream=stream, raise_on_error=False)
            torch.cuda.synchronize()
            st["wall_s"] = time.perf_counter() - t4
            st["mie_rel_l2"] = mie_err(xs)
            if args.solve_m2l_tensor == 3:
                # the same preconditioned solve with the 3xTF32 outer residual
                xs3 = torch.zeros_like(b)
                t7 = time.perf_counter()
                st3 = fdbem.bm_fgmres_solve(S2.plan, pc, net, b, xs3, tol=0.95e-5, restart=100, max_iter=2000,
                                            refine=True, inner_tol=1e-3, stream=stream, raise_on_error=False,
                                            refine_residual=1)
                torch.cuda.synchronize()
                st3["wall_s"] = time.perf_counter() - t7
                st3["mie_rel_l2"] = mie_err(xs3)
                st3["rel_residual_fp64"] = fp64_residual(S2, b, xs3)
                solve_alt["mixed_leaf_precond_3xtf32_residual"] = st3
            st["train_s"] = train_s
            st["training"] = tinfo
            # the network's weights are kept only if training beat its start, the exact leaf-block solution
            # (block Jacobi); the entry says which weights ran
            st["weights"] = "trained network" if tinfo.get("kept") == "trained" else "leaf-block solution (block Jacobi)"
            solve_alt["mixed_leaf_precond"] = st
            fdbem.bm_precond_destroy(pc)
            fdbem.bm_net_destroy(net)
        if puls is not None:
            # closed form of Sec. 5.2 for radius a: u = a/(1 - ika) on the surface (n into the body)
            a_s = spec.get("radius", 0.5)
            ue = a_s / complex(1.0, -k * a_s)
            up = torch.zeros_like(b_puls)
            t6 = time.perf_counter()
            st = fdbem.bm_gmres_solve(S2.plan, b_puls, up, tol=1e-5, restart=100, max_iter=2000, refine=True,
                                      inner_tol=1e-3, stream=stream, raise_on_error=False)
            torch.cuda.synchronize()
            uh = up.cpu().numpy()
            puls.update(st)
            puls.update({"wall_s": time.perf_counter() - t6, "u_exact": [ue.real, ue.imag],
                         "max_rel_err": float(np.max(np.abs(uh - ue)) / abs(ue)),
                         "mean_rel_err": float(abs(np.mean(uh) - ue) / abs(ue)),
                         "rms_rel_err": float(np.sqrt(np.mean(np.abs(uh - ue) ** 2)) / abs(ue))})
        if args.batch > 1:
            batched = run_batched(S2, args, N, dev, stream, solve_alt.get("mixed"), fdbem, torch)
        S2.close()
    table1 = None
    if rank == 0 and not args.no_table1_sample:
        # the paper's own FDA benchmark (Table 1), one size: N = 294,912 points, k = 16 pi, eps = 1e-4
        table1 = table1_case(294912, 16 * math.pi, 1e-4, fdbem, torch, dev, stream, tune=not args.no_tune)
    peaks, peak_src = _peaks()
    p64, p32 = fdbem.fda_device_peaks()
    # roofline of the dominant phase of the mixed-precision matvec
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25  # measured bf16 x the nominal TF32/BF16 ratio
    bytes_near = 8.0 * (info["near_entries"] + info["corr_entries"]) + 4.0 * info["corr_entries"]
    # the near-field matrices stream once per pass of rpp right-hand sides
    rpp = tune_main["near_rhs_per_pass"] if tune_main else (1 if nrhs == 1 else (16 if nrhs >= 12 else 4))
    near_passes = -(-nrhs // rpp)
    near_sched = tune_main["near_split"] if tune_main else (1 if rpp == 16 else args.near_split)
    near_split = near_sched >= 1
    near_kernel = (f"k_near_stream<float2, {rpp}>" + (" after k_near_corr" if near_split else "")
                   + (" (double-buffered windows)" if near_sched == 2 or rpp == 16 else ""))
    near_gbs = bytes_near * near_passes / (ph32["near"] * 1e-3) / 1e9
    dom = max((p for p in ph32 if p not in ("perm", "assemble")), key=lambda p: ph32[p])
    dom_ms = ph32[dom]
    if dom == "near" and rpp > 1:
        # several right-hand sides per pass over the matrices: 8 flops per complex entry and right-hand side on
        # the FP32 FMA pipes
        achieved = 8.0 * (info["near_entries"] + info["corr_entries"]) * nrhs / (ph32["near"] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": p32, "unit": "TFLOP/s", "frac": achieved / p32,
                "traffic": None, "kernel": near_kernel,
                "peak_source": "FP32 FMA throughput measured on this GPU by fda_device_peaks"}
    elif dom == "near":
        achieved = near_gbs
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": near_kernel,
                "peak_source": f"{peak_src} hbm_gbs (copy, burst)"}
    elif dom == "m2l" and args.m2l_tensor == 1:
        achieved = info["flops_m2l"] * nrhs / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": tf32_peak, "unit": "TFLOP/s",
                "frac": achieved / tf32_peak, "traffic": None, "kernel": "k_m2l_tc3 (TF32 tcgen05)",
                "peak_source": f"{peak_src} bf16_tflops x 1.1/2.25 (nominal TF32/BF16)"}
    elif dom in ("m2l", "m2m", "l2l"):
        fl = info["flops_m2l"] if dom == "m2l" else info["flops_m2m_l2l"] / 2
        achieved = fl * nrhs / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": p32, "unit": "TFLOP/s", "frac": achieved / p32,
                "traffic": None, "kernel": f"k_{dom}<float2>",
                "peak_source": "FP32 FMA throughput measured on this GPU by fda_device_peaks"}
    else:
        bts = info["bytes_s2m_l2t"] / 2 / 2
        achieved = bts / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": f"k_{dom}<float2>",
                "peak_source": f"{peak_src} hbm_gbs"}
    roof["phase_ms"] = dom_ms
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(mesh, k, X if nrhs == 1 else X[0], args.cpu_rows)
    value = job_throughput(ws, nrhs, ms32)
    line = {
        "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": workload_config(args, spec, mesh, ws),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": job_throughput(ws, nrhs, e2e_ms), "unit": "matvec/s",
                "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
                "d2h_bytes_per_step": int(yh.numel() * yh.element_size())},
        "gpu_launches": launches * args.steps,
        "clocks": clocks.summary(local),
        "fp64": {"matvec_per_s": 1000.0 / ms64, "ms_per_matvec": ms64, "phase_ms": ph64},
        "mixed": {"matvec_per_s": 1000.0 / ms32, "ms_per_matvec": ms32, "phase_ms": ph32,
                  "schedule": ["serial", "two streams, near field at 2 CTAs/SM",
                               "two streams, near field at 1 CTA/SM", "two streams, near field at 3 CTAs/SM"][overlap]
                  + (", near-field matrices evict-first in L2" if evict else "")
                  + (", M2L levels on concurrent streams" if farp else ""),
                  "phase_note": "phase_ms come from one serial product with an event between phases"},
        "speedup_matvec_mixed_vs_fp64": ms64 / ms32,
        "near_field": {"kernel": near_kernel, "ms": ph32["near"], "achieved_gbs": near_gbs,
                       "peak_gbs": peaks["hbm_gbs"], "frac": near_gbs / peaks["hbm_gbs"],
                       "algorithmic_bytes": bytes_near * near_passes, "passes": near_passes,
                       "rhs_per_pass": rpp, "corrections_split": near_split},
        "m2l_tensor": args.m2l_tensor,
        "autotune": tune_main,
        "batched": batched,
        "table1_sample": table1,
        "pulsating_sphere": puls,
        "solve_alpha_i_over_k": solve,
        "solve_alpha_minus_i_over_k": solve_alt,
        "speedup_solve_mixed_vs_fp64": (solve_alt["fp64"]["wall_s"] / solve_alt["mixed"]["wall_s"])
        if solve_alt else None,
        "speedup_solve_mixed_leaf_precond_vs_fp64": (solve_alt["fp64"]["wall_s"] /
                                                     solve_alt["mixed_leaf_precond"]["wall_s"])
        if solve_alt.get("mixed_leaf_precond") else None,
        "speedup_solve_mixed_3xtf32_residual_vs_fp64": (solve_alt["fp64"]["wall_s"] /
                                                        solve_alt["mixed_3xtf32_residual"]["wall_s"])
        if solve_alt.get("mixed_3xtf32_residual") else None,
        "speedup_solve_mixed_3xtf32_residual_fp64_check_vs_fp64": (
            solve_alt["fp64"]["wall_s"] / solve_alt["mixed_3xtf32_residual_fp64_check"]["wall_s"])
        if solve_alt.get("mixed_3xtf32_residual_fp64_check") else None,
        "speedup_solve_mixed_leaf_precond_3xtf32_residual_vs_fp64": (
            solve_alt["fp64"]["wall_s"] / solve_alt["mixed_leaf_precond_3xtf32_residual"]["wall_s"])
        if solve_alt.get("mixed_leaf_precond_3xtf32_residual") else None,
        "measured_fma_tflops": {"fp64": p64, "fp32": p32},
        "setup_s": setup_s, "setup_ms": info["setup_ms"],
        "plan": {k_: info[k_] for k_ in ("lmin", "n_leaves", "n_direct_blocks", "near_entries", "corr_entries",
                                         "flops_m2l", "flops_m2m_l2l", "bytes_near", "bytes_s2m_l2t",
                                         "device_bytes")},
        "levels": {str(l): {"s": info["s"][l], "wedges": info["n_wedges"][l], "pairs": info["m2l_pairs"][l],
                            "offsets": info["m2l_offsets"][l], "lowrank": info["m2l_lowrank"][l],
                            "m2l_gflops": info["m2l_flops_lev"][l] / 1e9,
                            "m2l_op_bytes_fp32": info["m2l_op_bytes_lev"][l] / 2}
                   for l in range(32) if info["s"][l] > 0},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
