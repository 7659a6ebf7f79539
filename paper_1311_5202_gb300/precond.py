"""Training and use of the learned leaf-block preconditioner (flexible GMRES).

Training pairs come from the method's own solves: for a right-hand side b, a converged GMRES solve gives
x*; restarted GMRES cycles from x = 0 give iterates x_k, and each yields a residual/correction pair
r_k = b - A x_k, e_k = x* - x_k (A e_k = r_k). The network is trained on the GPU (hand-written forward,
backward and Adam kernels in the library) to map residuals to corrections; in flexible GMRES it is the
right preconditioner. Every arithmetic step runs in the CUDA library; this module only orchestrates.
"""
from __future__ import annotations

import numpy as np

from . import fdbem


def net_init(net, mode="block"):
    """Set the output layer: "identity" (z = r) or "block" (z = y = A_LL^-1 r, the leaf block solution)."""
    w = fdbem.bm_net_params(net)
    n = w.size
    H = int(round((-12 + np.sqrt(128 + 4 * n)) / 2))  # n = 6H + H + H^2 + H + 4H + 4 = H^2 + 12H + 4
    W3 = 6 * H + H + H * H + H
    w[W3:W3 + 4 * H] = 0.0
    w[W3 + 4 * H:] = [1, 0, 0, 0] if mode == "identity" else [0, 0, 1, 0]
    fdbem.bm_net_params(net, w)
    return net


def harvest(solver, dirs, restart=20, cycles=6, ref_tol=1e-7, stream=None):
    """Residual/correction pairs (R, E), each (npairs, N) complex128 on the device."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    N = solver.N
    R, E = [], []
    for d in np.atleast_2d(dirs):
        b = torch.empty(N, dtype=torch.complex128, device=dev)
        fdbem.bm_rhs_plane_wave(solver.prob, d, b, stream)
        xs = torch.zeros_like(b)
        fdbem.bm_gmres_solve(solver.plan, b, xs, tol=ref_tol, restart=300, max_iter=3000, stream=stream,
                             raise_on_error=False)
        x = torch.zeros_like(b)
        for _ in range(cycles):
            fdbem.bm_gmres_solve(solver.plan, b, x, tol=1e-14, restart=restart, max_iter=restart, x0_given=True,
                                 stream=stream, raise_on_error=False)
            r = torch.empty_like(b)
            e = torch.empty_like(b)
            fdbem.bm_residual_pair(solver.plan, b, xs, x, r, e, stream)
            R.append(r)
            E.append(e)
    return torch.stack(R), torch.stack(E)


def train(net, datasets, epochs=30, lr=3e-3, batch=4, stream=None, log=None):
    """datasets: list of (precond, R, E). Adam over mini-batches of pairs; returns the loss history."""
    import torch
    hist = []
    rng = np.random.default_rng(0)
    for ep in range(epochs):
        tot, cnt = 0.0, 0
        for pc, R, E in datasets:
            order = rng.permutation(R.shape[0])
            for s in range(0, len(order), batch):
                idx = torch.as_tensor(order[s:s + batch], device=R.device)
                loss, _ = fdbem.bm_precond_train_step(pc, net, R[idx].contiguous(), E[idx].contiguous(), lr=lr,
                                                      stream=stream)
                tot += loss
                cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


def select(solver, pc, candidates, dirs, tol=1e-5, restart=100, max_iter=2000, stream=None):
    """Judge candidate parameter sets by the iterations flexible GMRES needs on a held-out problem and keep
    the best one (returns its index and the iteration counts)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    counts = []
    for net in candidates:
        it = 0
        for d in np.atleast_2d(dirs):
            b = torch.empty(solver.N, dtype=torch.complex128, device=dev)
            fdbem.bm_rhs_plane_wave(solver.prob, d, b, stream)
            x = torch.zeros_like(b)
            st = fdbem.bm_fgmres_solve(solver.plan, pc, net, b, x, tol=tol, restart=restart, max_iter=max_iter,
                                       stream=stream, raise_on_error=False)
            it += st["iterations"] if st["status"] == 0 else max_iter
        counts.append(it)
    return int(np.argmin(counts)), counts


def build_trained(train_meshes, alpha_sign=-1, hidden=32, seed=7, eps=1e-4, epochs=25, lr=2e-3, log=None,
                  dirs_per_mesh=6, stream=None):
    """Train a network on the given meshes ((mesh, k) pairs): harvest pairs from the method's own GMRES
    solves, start at the block solution, train, and keep the trained weights only if they cut the flexible
    GMRES iterations on the last (held-out) mesh. Returns (net, info)."""
    solvers, datasets = [], []
    try:
        for mesh, k in train_meshes:
            S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=eps, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                             alpha=alpha_sign * 1j / k)
            pc = fdbem.bm_precond_create(S.plan)
            solvers.append((S, pc))
        from .inputs import fibonacci_directions
        for S, pc in solvers[:-1]:
            R, E = harvest(S, fibonacci_directions(dirs_per_mesh), stream=stream)
            datasets.append((pc, R, E))
        start = net_init(fdbem.bm_net_create(hidden, seed), "block")
        net = net_init(fdbem.bm_net_create(hidden, seed), "block")
        hist = train(net, datasets, epochs=epochs, lr=lr, stream=stream, log=log)
        Sv, pcv = solvers[-1]
        best, counts = select(Sv, pcv, [start, net], fibonacci_directions(2), stream=stream)
        keep, drop = (start, net) if best == 0 else (net, start)
        fdbem.bm_net_destroy(drop)
        return keep, dict(loss_first=hist[0], loss_last=hist[-1], validation_iterations=counts,
                          kept="trained" if best == 1 else "block start")
    finally:
        for S, pc in solvers:
            fdbem.bm_precond_destroy(pc)
            S.close()


def compare(solver, pc, net, dirs, tol=1e-5, restart=100, max_iter=3000, stream=None):
    """Iterations and times to tol: GMRES without preconditioner vs flexible GMRES with the network."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    out = []
    for d in np.atleast_2d(dirs):
        b = torch.empty(solver.N, dtype=torch.complex128, device=dev)
        fdbem.bm_rhs_plane_wave(solver.prob, d, b, stream)
        x0 = torch.zeros_like(b)
        s0 = fdbem.bm_gmres_solve(solver.plan, b, x0, tol=tol, restart=restart, max_iter=max_iter, stream=stream,
                                  raise_on_error=False)
        x1 = torch.zeros_like(b)
        s1 = fdbem.bm_fgmres_solve(solver.plan, pc, net, b, x1, tol=tol, restart=restart, max_iter=max_iter,
                                   stream=stream, raise_on_error=False)
        out.append((s0, s1))
    return out
