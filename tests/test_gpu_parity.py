"""GPU path vs the FP64 oracle, through the C ABI (rows a1-a13 of the hot path).

Tolerances: tree and lists bit-exact; geometry to rounding; corrections to 1e-8 of the row scale
(the two sides use different quadrature orders); FDA matvec relative l2 <= 1e-4 (FP64 path) and
<= 3e-4 (FP32 path); solution within 1e-4 of the oracle's direct solve, within the discretisation
error of the Mie series.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1311_5202_gb300 import fdbem, inputs  # noqa: E402

DEV = "cuda:0"


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def c1():
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    S = fdbem.Solver(mesh.nodes, mesh.elems, 10.0, eps=1e-6, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     nrhs_max=4)
    yield mesh, S
    S.close()


# ------------------------------------------------------------------ a1 geometry
def test_nystrom_geometry_matches_oracle(c1):
    mesh, S = c1
    N = S.N
    x = torch.empty(N * 3, dtype=torch.float64, device=DEV)
    n = torch.empty(N * 3, dtype=torch.float64, device=DEV)
    w = torch.empty(N, dtype=torch.float64, device=DEV)
    fdbem.bm_problem_geometry(S.prob, x, n, w)
    xo, no, wo = O.geometry(mesh.nodes, mesh.elems)
    # the point formula is evaluated in the same operation order without contraction on both sides
    assert np.array_equal(x.cpu().numpy().reshape(N, 3), xo)
    assert np.array_equal(n.cpu().numpy().reshape(N, 3), no)
    assert np.array_equal(w.cpu().numpy(), wo)


# ------------------------------------------------------------------ a2, a3 tree + lists, bit-exact
TREE_CASES = [
    ("sphere_k10_leaf64", lambda: inputs.icosphere(4, 0.5), 64, 10.0),
    ("sphere_k100_leaf16", lambda: inputs.icosphere(5, 0.5), 16, 100.0),
    ("spheroid_k60_leaf24", lambda: inputs.ellipsoid(6, (1.0, 0.25, 0.25)), 24, 60.0),
    ("torus_k40_leaf20", lambda: inputs.torus(0.5, 0.2, 24, 10), 20, 40.0),
    ("sphere_k100_leaf64_N100k", lambda: inputs.icosphere(29, 0.5), 64, 100.0),
]


@pytest.mark.parametrize("name,mk,leaf,k", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_and_lists_bit_exact(name, mk, leaf, k):
    _need_gpu()
    mesh = mk()
    prob = fdbem.bm_problem_create(mesh.nodes, mesh.elems, k)
    try:
        tree = fdbem.fda_build_tree(prob, leaf)
        try:
            G = fdbem.fda_tree_export(tree)
        finally:
            fdbem.fda_tree_destroy(tree)
    finally:
        fdbem.bm_problem_destroy(prob)
    xo, _, _ = O.geometry(mesh.nodes, mesh.elems)
    R = O.tree(xo, leaf, k)
    assert np.array_equal(G["corner"], R["corner"]) and G["side"] == R["side"]
    for key in ("perm", "keys", "level", "ix", "iy", "iz", "nchild", "leaf", "parent", "child_begin", "pbeg", "pend",
                "lev_hf", "lev_T", "lev_n", "direct", "m2l_tgt", "m2l_src", "m2l_level", "m2l_off", "m2l_wout",
                "m2l_win"):
        assert np.array_equal(G[key], R[key]), key


# ------------------------------------------------------------------ a5 corrections
def test_near_corrections_match_oracle(c1):
    mesh, S = c1
    k = 10.0
    rows = inputs.sample_rows(S.N, 48, 11)
    got = fdbem.fda_corrections_export(S.plan, rows)
    ref = O.correction_weights(mesh.nodes, mesh.elems, k, rows)
    xs, ns, ws = O.geometry(mesh.nodes, mesh.elems)
    alpha = 1j / k
    for r, i in enumerate(rows):
        elist, wD, wH = ref[r]
        cols = (6 * elist[:, None] + np.arange(6)[None, :]).ravel()
        wbar = (wD + alpha * wH).ravel()
        kk = O.kernels(np.repeat(xs[i:i + 1], len(cols), 0), np.repeat(ns[i:i + 1], len(cols), 0), xs[cols],
                       ns[cols], k)
        direct = (kk[:, 1] + alpha * kk[:, 3]) * ws[cols]
        direct[cols == i] = 0
        cref = wbar - direct
        gc, gv = got[r]
        assert np.array_equal(np.sort(gc), np.sort(cols)), i
        order = np.argsort(gc)
        scale = np.max(np.abs(cref))
        assert np.max(np.abs(gv[order] - cref[np.argsort(cols)])) < 1e-8 * scale, i


# ------------------------------------------------------------------ a6-a12 matvec
def _oracle_rows(mesh, k, x, rows):
    return O.matvec_rows(mesh.nodes, mesh.elems, k, x, rows)


def test_fda_matvec_fp64_matches_dense_oracle_all_rows(c1):
    mesh, S = c1
    x = inputs.complex_gaussian(S.N, 20131120)
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty_like(xd)
    # the FP32 plan keeps its FP64 operators: run the plain FP64 product explicitly
    fdbem.fda_matvec_ex(S.plan, fdbem.FDA_PREC_FP64, xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    rows = np.arange(S.N)
    yo = _oracle_rows(mesh, 10.0, x, rows)
    err = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    assert err < 1e-4, err


def test_fda_matvec_fp32_path(c1):
    mesh, S = c1
    x = inputs.complex_gaussian(S.N, 5)
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty_like(xd)
    S.matvec(xd, yd)
    torch.cuda.synchronize()
    rows = inputs.sample_rows(S.N, 256, 7)
    yo = _oracle_rows(mesh, 10.0, x, rows)
    err = np.linalg.norm(yd.cpu().numpy()[rows] - yo) / np.linalg.norm(yo)
    assert err < 3e-4, err


def test_matvec_batched_rhs_equals_single(c1):
    mesh, S = c1
    X = inputs.complex_gaussian(S.N, 9, nrhs=3)
    Xd = torch.from_numpy(X).to(DEV).contiguous()
    Yd = torch.empty_like(Xd)
    S.matvec(Xd, Yd)
    for r in range(3):
        y1 = torch.empty_like(Xd[r])
        S.matvec(Xd[r].contiguous(), y1)
        torch.cuda.synchronize()
        a, b = Yd[r].cpu().numpy(), y1.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-6


@pytest.mark.parametrize("split,form", [(1, 0), (2, 0), (0, 1), (1, 1), (2, 1), (2, 2), (1, 2), (2, 3)])
def test_near_correction_split_schedule(c1, split, form):
    """The off-block correction entries of Eq. kcorrection as their own CSR kernel before the near-field stream
    (near_split = 1), and with the stream's density windows double-buffered (near_split = 2); each schedule also
    with the four-stage ring of one right-hand side (form 1), and the double-buffered one with packed FP32x2 FMAs
    on duplicated densities (form 2) and in the slim CTA (form 3; both FP32 products only): the FP64 product on
    all rows against the oracle
    (1e-4), and against the per-leaf schedule of the same plan (same sums in another order: 1e-12 in FP64, 1e-5
    in FP32); for split = 1 also 16 right-hand sides (the 16-wide pass reduces lane sums by recursive halving and
    always double-buffers its windows; with form 2 it pairs each matrix entry in registers for packed FMAs)."""
    mesh, S0 = c1
    S1 = fdbem.Solver(mesh.nodes, mesh.elems, 10.0, eps=1e-6, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                      nrhs_max=16, near_split=split, near_form=form)
    try:
        x = inputs.complex_gaussian(S1.N, 77)
        xd = torch.from_numpy(x).to(DEV)
        y1, y0 = torch.empty_like(xd), torch.empty_like(xd)
        fdbem.fda_matvec_ex(S1.plan, fdbem.FDA_PREC_FP64, xd, y1)
        fdbem.fda_matvec_ex(S0.plan, fdbem.FDA_PREC_FP64, xd, y0)
        torch.cuda.synchronize()
        a, b = y1.cpu().numpy(), y0.cpu().numpy()
        yo = _oracle_rows(mesh, 10.0, x, np.arange(S1.N))
        assert np.linalg.norm(a - yo) / np.linalg.norm(yo) < 1e-4
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
        x32 = torch.from_numpy(x.astype(np.complex64)).to(DEV)
        z1, z0 = torch.empty_like(x32), torch.empty_like(x32)
        S1.matvec(x32, z1)
        S0.matvec(x32, z0)
        torch.cuda.synchronize()
        g, h = z1.cpu().numpy(), z0.cpu().numpy()
        assert np.linalg.norm(g - h) / np.linalg.norm(h) < 1e-5
        if split == 1:
            X = inputs.complex_gaussian(S1.N, 78, nrhs=16)
            Xd = torch.from_numpy(X.astype(np.complex64)).to(DEV).contiguous()
            Y1 = torch.empty_like(Xd)
            S1.matvec(Xd, Y1)
            torch.cuda.synchronize()
            rows = inputs.sample_rows(S1.N, 64, 79)
            for r in (0, 7, 15):
                y0r = torch.empty_like(Xd[r])
                S0.matvec(Xd[r].contiguous(), y0r)
                torch.cuda.synchronize()
                g, h = Y1[r].cpu().numpy(), y0r.cpu().numpy()
                assert np.linalg.norm(g - h) / np.linalg.norm(h) < 1e-5, r
                yo = _oracle_rows(mesh, 10.0, X[r].astype(np.complex128), rows)
                assert np.linalg.norm(g[rows] - yo) / np.linalg.norm(yo) < 3e-4, r
        assert fdbem.fda_plan_check(S1.plan) == fdbem.FDA_OK
    finally:
        S1.close()


@pytest.mark.parametrize("nrhs", [13, 17])
def test_ragged_wide_batches_equal_single_products(c1, nrhs):
    """Ragged passes of the 16-wide near field: 13 right-hand sides (one pass with 3 zero-filled lanes) and 17
    (a full pass, then a pass of one), odd counts that take the 8-byte density copies. Every right-hand side
    equals its own single product to FP32 rounding (1e-5; the two use different near-field kernels and
    summation orders)."""
    mesh, S0 = c1
    S = fdbem.Solver(mesh.nodes, mesh.elems, 10.0, eps=1e-6, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     nrhs_max=nrhs)
    try:
        X = inputs.complex_gaussian(S.N, 300 + nrhs, nrhs=nrhs).astype(np.complex64)
        Xd = torch.from_numpy(X).to(DEV).contiguous()
        Yd = torch.empty_like(Xd)
        S.matvec(Xd, Yd)
        torch.cuda.synchronize()
        for r in sorted({0, 11, 12, nrhs - 1}):
            y1 = torch.empty_like(Xd[r])
            S0.matvec(Xd[r].contiguous(), y1)
            torch.cuda.synchronize()
            a, b = Yd[r].cpu().numpy(), y1.cpu().numpy()
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, r
        assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK
    finally:
        S.close()


# ------------------------------------------------------------------ a13 solve
def test_gmres_solve_matches_oracle_and_mie(c1):
    mesh, S = c1
    k = 10.0
    b = torch.empty(S.N, dtype=torch.complex128, device=DEV)
    fdbem.bm_rhs_plane_wave(S.prob, [0.0, 0.0, 1.0], b)
    xs, ns, ws = O.geometry(mesh.nodes, mesh.elems)
    bo = O.bm_rhs(xs, ns, k, [0, 0, 1])
    assert np.allclose(b.cpu().numpy(), bo, rtol=1e-13, atol=1e-14)
    x = torch.zeros_like(b)
    st = S.solve(b, x, tol=1e-6, restart=50, max_iter=300)
    assert st["rel_residual"] <= 1e-6
    A = O.dense_matrix(mesh.nodes, mesh.elems, k)
    xo = np.linalg.solve(A, bo)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-4
    th = np.arccos(np.clip(xs[:, 2] / np.linalg.norm(xs, axis=1), -1, 1))
    mie = O.mie_total_surface(th, k, 0.5)
    # 320 elements (h ~ lambda/4.5): the discretisation error against the Mie series is 5.1e-3 here, the
    # same as the oracle's own dense solve; the 1e-3 bar is met on the refined mesh below
    assert np.linalg.norm(xg - mie) / np.linalg.norm(mie) < 6e-3


def _mie(xs, k, a, chunk=200000):
    th = np.arccos(np.clip(xs[:, 2] / np.linalg.norm(xs, axis=1), -1, 1))
    return np.concatenate([O.mie_total_surface(th[i:i + chunk], k, a) for i in range(0, len(th), chunk)])


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_mie_refined_sphere_within_1e3(form):
    """Sec. 5.3, rigid-sphere scattering of u_inc = e^{ikz} at kD = 10 on 2000 curved elements (12,000 DOF,
    h ~ lambda/7): the library's GMRES solution (plain FP64, and the mixed form: FP32 near field, TF32
    tensor-core translations, FP64 refinement) is within 1e-3 of the Mie series in relative l2."""
    _need_gpu()
    mesh = inputs.icosphere(10, 0.5)
    k = 10.0
    if form == "fp64":
        S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64)
    else:
        S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                         m2l_tensor=1)
    try:
        b = torch.empty(S.N, dtype=torch.complex128, device=DEV)
        fdbem.bm_rhs_plane_wave(S.prob, [0.0, 0.0, 1.0], b)
        x = torch.zeros_like(b)
        if form == "fp64":
            st = S.solve(b, x, tol=1e-7, restart=50, max_iter=400)
        else:
            st = S.solve(b, x, tol=1e-7, restart=50, max_iter=600, refine=True, inner_tol=1e-3)
        assert st["rel_residual"] <= 1e-7
        xs, _, _ = O.geometry(mesh.nodes, mesh.elems)
        mie = _mie(xs, k, 0.5)
        err = np.linalg.norm(x.cpu().numpy() - mie) / np.linalg.norm(mie)
        assert err < 1e-3, (form, err)
    finally:
        S.close()


def test_refinement_solve_fp32_inner(c1):
    mesh, S = c1
    b = torch.empty(S.N, dtype=torch.complex128, device=DEV)
    fdbem.bm_rhs_plane_wave(S.prob, [1.0, 0.0, 0.0], b)
    x = torch.zeros_like(b)
    st = S.solve(b, x, tol=1e-6, restart=50, max_iter=400, refine=True, inner_tol=1e-3)
    assert st["rel_residual"] <= 1e-6 and st["outer_iterations"] >= 1


# ------------------------------------------------------------------ high-frequency levels (directional wedges)
@pytest.mark.parametrize("form", ["fp64", "tensor"])
def test_fda_matvec_with_directional_levels_sampled_rows(form):
    """kD = 100 sphere with directional (wedge) levels: the FP64 form (<= 1e-4) and the mixed form with M2L,
    M2M and L2L on the TF32 tensor cores (<= 3e-4), two right-hand sides, against the oracle's rows."""
    _need_gpu()
    mesh = inputs.icosphere(14, 0.5)
    k = 100.0
    if form == "fp64":
        S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=64, nrhs_max=2)
    else:
        S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                         m2l_tensor=1, nrhs_max=2)
    try:
        info = S.info()
        assert any(info["n_wedges"][l] > 1 and info["m2l_pairs"][l] > 0 for l in range(32))
        x = inputs.complex_gaussian(S.N, 20131120, nrhs=2)
        xd = torch.from_numpy(x).to(DEV).contiguous()
        yd = torch.empty_like(xd)
        S.matvec(xd, yd)
        torch.cuda.synchronize()
        rows = inputs.sample_rows(S.N, 256, 7)
        for r in range(2):
            yo = _oracle_rows(mesh, k, x[r], rows)
            err = np.linalg.norm(yd[r].cpu().numpy()[rows] - yo) / np.linalg.norm(yo)
            assert err < (1e-4 if form == "fp64" else 3e-4), (form, r, err)
    finally:
        S.close()


@pytest.mark.parametrize("form", ["fp64", "mixed", "mixed3"])
def test_bm_operator_with_two_directional_levels(form):
    """The Burton-Miller product with M2L pairs on two high-frequency levels, so that the nested-wedge
    M2M and L2L (24 wedges at level 4, 6 at level 5) carry the far field: a coarse sphere at k = 300
    (kD = 300, 48,000 DOF, 16 points per leaf), eps = 1e-5. FP64 form (<= 1e-4) and the FP32 form (FP32 near
    field and FP32 translations, <= 3e-4) on 256 oracle rows. (At this geometry the FP64 error follows eps at
    about 1.8 eps: 1.8e-4, 1.9e-5, 1.7e-6 for eps = 1e-4, 1e-5, 1e-6, with or without the low-rank
    translations. The far field carries most of this product, so TF32 translations, whose gathered operands
    the tensor cores truncate to 10 mantissa bits, land at 6.4e-4.) The form "mixed3" is the FP32 form with
    3xTF32 tensor-core translations (m2l_tensor = 3), autotuned, at the same 3e-4 bar."""
    _need_gpu()
    mesh = inputs.icosphere(20, 0.5)
    k = 300.0
    if form == "fp64":
        S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=16)
    else:
        S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=16, precision=fdbem.FDA_PREC_FP32,
                         m2l_tensor=3 if form == "mixed3" else 0)
    try:
        info = S.info()
        hf_m2l = [l for l in range(32) if info["n_wedges"][l] > 1 and info["m2l_pairs"][l] > 0]
        assert len(hf_m2l) >= 2, hf_m2l
        assert max(info["n_wedges"][l] for l in hf_m2l) >= 24
        if form == "mixed3":
            fdbem.fda_autotune(S.plan, 1)
        x = inputs.complex_gaussian(S.N, 20131120)
        xd = torch.from_numpy(x).to(DEV)
        yd = torch.empty_like(xd)
        S.matvec(xd, yd)
        torch.cuda.synchronize()
        rows = inputs.sample_rows(S.N, 256, 7)
        yo = _oracle_rows(mesh, k, x, rows)
        err = np.linalg.norm(yd.cpu().numpy()[rows] - yo) / np.linalg.norm(yo)
        assert err < (1e-4 if form == "fp64" else 3e-4), (form, err)
        assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK
    finally:
        S.close()


def test_tiny_mesh_without_far_field():
    """Every pair is near: the plan has no translations and the matvec is the corrected direct sum."""
    _need_gpu()
    mesh = inputs.icosphere(1, 0.5)  # 20 elements, 120 DOF < leaf size
    S = fdbem.Solver(mesh.nodes, mesh.elems, 3.0, eps=1e-6, leaf_max=200)
    try:
        x = inputs.complex_gaussian(S.N, 3)
        xd = torch.from_numpy(x).to(DEV)
        yd = torch.empty_like(xd)
        S.matvec(xd, yd)
        torch.cuda.synchronize()
        yo = _oracle_rows(mesh, 3.0, x, np.arange(S.N))
        assert np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo) < 1e-10
    finally:
        S.close()


# ------------------------------------------------------------------ tensor-core M2L (tcgen05)
@pytest.mark.parametrize("split", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13])
def test_tensor_core_selftest(split):
    """A complex operator applied to gathered columns on the tensor cores against an FP64 host product (TF32:
    ~1e-4 of the row scale; 3xTF32 split: FP32 level). split 2..5 is the pre-expanded-image kernel in its four
    tile shapes with M = min(256, K) rows: K = 8, 37 (one 128-row tile, ragged K), 111 (two tiles), 222 (four
    tiles); 6, 7 the same kernel with the bulk-reduction epilogue; 8, 9 the swapped-operand V^ kernel
    (M = min(100, K): 32, 128 and 256 TMEM columns, one and two operator tiles); 10, 11 3xTF32 from the TF32
    and remainder images (FP32 level); 12, 13 the swapped kernel with 16-wide K chunks."""
    _need_gpu()
    for K in ((16, 111, 222) if split < 2 else (8, 37, 111, 222)):
        err, wait_failed = fdbem.fda_tc_selftest(K, split)
        assert wait_failed == 0
        assert err < (5e-6 if split in (1, 10, 11) else 1e-3), (K, err)


@pytest.mark.parametrize("mode", [1, 2])
def test_fda_matvec_tensor_core_m2l(mode):
    """FP32 plan with M2L on the tensor cores (TF32 from pre-expanded operator images, or 3xTF32 split)
    against the dense oracle (<= 3e-4), two right-hand sides."""
    _need_gpu()
    mesh = inputs.icosphere(8, 0.5)
    k = 20.0
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     m2l_tensor=mode, nrhs_max=2)
    try:
        x = inputs.complex_gaussian(S.N, 5, nrhs=2)
        xd = torch.from_numpy(x).to(DEV).contiguous()
        yd = torch.empty_like(xd)
        S.matvec(xd, yd)
        torch.cuda.synchronize()
        rows = inputs.sample_rows(S.N, 200, 7)
        for r in range(2):
            yo = _oracle_rows(mesh, k, x[r], rows)
            err = np.linalg.norm(yd[r].cpu().numpy()[rows] - yo) / np.linalg.norm(yo)
            assert err < 3e-4, (mode, r, err)
    finally:
        S.close()


@pytest.fixture(scope="module")
def kd100_variants():
    """kD = 100 sphere (23,520 DOF) with one directional level and three low-frequency levels; FP32 plan with
    the TF32 operator images; three right-hand sides and their oracle rows."""
    _need_gpu()
    mesh = inputs.icosphere(14, 0.5)
    k = 100.0
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     m2l_tensor=1, nrhs_max=3)
    x = inputs.complex_gaussian(S.N, 41, nrhs=3)
    rows = inputs.sample_rows(S.N, 256, 7)
    yo = [_oracle_rows(mesh, k, x[r], rows) for r in range(3)]
    xd = torch.from_numpy(x.astype(np.complex64)).to(DEV).contiguous()
    y0 = torch.empty_like(xd)
    S.matvec(xd, y0)
    torch.cuda.synchronize()
    yield S, xd, y0.cpu().numpy(), rows, yo
    S.close()


@pytest.mark.parametrize("variant", [0, 1, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15])
def test_forced_m2l_variants_match_oracle(kd100_variants, variant):
    """Every M2L kernel variant the autotuner may choose, forced for all levels and stages of one plan: FMA (0),
    TF32 operator images in four tile shapes (1, 3-5), the bulk-reduction epilogue (6, 7), the swapped-operand
    V^ kernel (8, 9), the persistent warp-specialised U^ kernel (10, with 8 for the V^ stage), the narrow
    bulk-reduction shape with exact row tiles (11), the V^ kernel fed by TMA row gathers (12, 13; with three
    right-hand sides it falls back to 8, so a one-column product is checked too), the swapped V^ kernel with
    16-wide K chunks (14, 15). Each product
    meets the mixed bar on 256 oracle rows for three right-hand sides. The
    tensor-core variants share their TF32 arithmetic and differ from the default one only in the order of the
    additions (2e-5); the FP32 FMA variant differs from it by the TF32 rounding of the translations (5e-4)."""
    S, xd, y0, rows, yo = kd100_variants
    fdbem.fda_m2l_force(S.plan, variant)
    try:
        yd = torch.empty_like(xd)
        S.matvec(xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        for r in range(3):
            err = np.linalg.norm(y[r][rows] - yo[r]) / np.linalg.norm(yo[r])
            assert err < 3e-4, (variant, r, err)
            bar = 5e-4 if variant == 0 else 2e-5
            assert np.linalg.norm(y[r] - y0[r]) / np.linalg.norm(y0[r]) < bar, (variant, r)
        if variant in (12, 13):  # the TMA-fed kernel runs for one right-hand side
            x1 = xd[0].contiguous()
            y1 = torch.empty_like(x1)
            S.matvec(x1, y1)
            torch.cuda.synchronize()
            g = y1.cpu().numpy()
            assert np.linalg.norm(g[rows] - yo[0]) / np.linalg.norm(yo[0]) < 3e-4
            assert np.linalg.norm(g - y0[0]) / np.linalg.norm(y0[0]) < 2e-5
        assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK
    finally:
        fdbem.fda_m2l_force(S.plan, -1)


def test_fp32_only_plan():
    """A plan that drops its FP64 operators (drop_fp64 = 1) keeps the mixed product (3e-4 against the oracle,
    and the same numbers as the plan that keeps both copies), refuses FP64 products and refinement with
    FDA_E_STATE, solves with GMRES around its FP32 operator, and holds less device memory. The translations
    are 3xTF32 here: GMRES on an operator whose translations round to TF32 stalls near a 1e-4 residual (the
    rounding makes the product slightly nonlinear), while FP32-level translations reach 1e-5."""
    _need_gpu()
    mesh = inputs.icosphere(14, 0.5)
    k = 100.0
    kw = dict(eps=1e-4, leaf_max=64, precision=fdbem.FDA_PREC_FP32, m2l_tensor=3, alpha=-1j / k)
    S1 = fdbem.Solver(mesh.nodes, mesh.elems, k, **kw)
    S2 = fdbem.Solver(mesh.nodes, mesh.elems, k, drop_fp64=True, **kw)
    try:
        i1, i2 = S1.info(), S2.info()
        assert i1["device_bytes"] - i2["device_bytes"] >= 16 * i1["near_entries"]  # at least the FP64 near field
        x = inputs.complex_gaussian(S1.N, 23)
        xd = torch.from_numpy(x.astype(np.complex64)).to(DEV)
        y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
        S1.matvec(xd, y1)
        S2.matvec(xd, y2)
        torch.cuda.synchronize()
        a, b = y2.cpu().numpy(), y1.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
        rows = inputs.sample_rows(S1.N, 128, 7)
        yo = O.matvec_rows(mesh.nodes, mesh.elems, k, x, rows, beta_h=-1j / k)
        assert np.linalg.norm(a[rows] - yo) / np.linalg.norm(yo) < 3e-4
        x64 = torch.from_numpy(x).to(DEV)
        rc = fdbem.lib().fda_matvec_ex(S2.plan, fdbem.FDA_PREC_FP64, fdbem.C.c_void_p(x64.data_ptr()),
                                        fdbem.C.c_void_p(torch.empty_like(x64).data_ptr()), 1, fdbem.FDA_CPLX128,
                                        None)
        assert rc == fdbem.FDA_E_STATE and "drop_fp64" in fdbem.fda_last_error()
        bb = torch.empty(S2.N, dtype=torch.complex128, device=DEV)
        fdbem.bm_rhs_plane_wave(S2.prob, [0.0, 0.0, 1.0], bb)
        u = torch.zeros_like(bb)
        st = S2.solve(bb, u, tol=1e-5, restart=100, max_iter=3000, refine=True, raise_on_error=False)
        assert st["status"] == fdbem.FDA_E_STATE
        st = S2.solve(bb, u, tol=1e-5, restart=100, max_iter=3000)
        assert st["status"] == fdbem.FDA_OK and st["rel_residual"] <= 1e-5
        # refinement with the 3xTF32 FP32 product as the outer residual needs no FP64 operator
        u3 = torch.zeros_like(bb)
        st = S2.solve(bb, u3, tol=1e-5, restart=100, max_iter=3000, refine=True, inner_tol=1e-3,
                      refine_residual=1)
        assert st["status"] == fdbem.FDA_OK and st["rel_residual"] <= 1e-5 and st["outer_iterations"] >= 1
        r = torch.empty_like(bb)
        fdbem.fda_matvec_ex(S1.plan, fdbem.FDA_PREC_FP64, u3, r)  # S1: the same operator with its FP64 copy
        torch.cuda.synchronize()
        assert (torch.linalg.norm(bb - r) / torch.linalg.norm(bb)).item() < 2e-5
        assert fdbem.fda_plan_check(S2.plan) == fdbem.FDA_OK
    finally:
        S2.close()
        S1.close()


# ------------------------------------------------------------------ lockstep block GMRES (several directions)
@pytest.mark.parametrize("refine", [False, True])
def test_block_gmres_several_directions_match_oracle(refine):
    """Three incident directions solved together (one block matvec per step, a Krylov space per column):
    every column meets the residual and matches the dense oracle solve of its own right-hand side."""
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    k = 10.0
    dirs = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 0.6, 0.8]])
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64,
                     precision=fdbem.FDA_PREC_FP32 if refine else fdbem.FDA_PREC_FP64, nrhs_max=3)
    try:
        b = torch.empty((3, S.N), dtype=torch.complex128, device=DEV)
        fdbem.bm_rhs_plane_wave(S.prob, dirs, b)
        x = torch.zeros_like(b)
        st = S.solve(b, x, tol=1e-6, restart=40, max_iter=400, refine=refine, inner_tol=1e-3)
        assert st["status"] == 0 and st["rel_residual"] <= 1e-6
        xs, ns, ws = O.geometry(mesh.nodes, mesh.elems)
        A = O.dense_matrix(mesh.nodes, mesh.elems, k)
        for c in range(3):
            xo = np.linalg.solve(A, O.bm_rhs(xs, ns, k, dirs[c]))
            xg = x[c].cpu().numpy()
            assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-4, c
    finally:
        S.close()


def test_tf32_pass_on_3xtf32_images_and_refinement_with_their_residual():
    """A plan with 3xTF32 images (m2l_tensor = 3) serves products in two arithmetics. FDA_PREC_FP32 runs the
    three-product split form; FDA_PREC_TF32 runs single-pass TF32 kernels on the leading part of the same images,
    the arithmetic of a TF32 plan (m2l_tensor = 1). Both meet the mixed bar (3e-4) on 256 oracle rows. The TF32
    pass agrees with the TF32 plan's product up to the rounding of the images (1e-4) and differs from the split
    form by more than FP32 rounding; an autotuned TF32 pass and a captured graph of it give the same product.
    Refinement with the split product as the outer residual (refine_residual = 1) reaches 1e-6 and, checked
    with the FP64 operator, 1e-5; it agrees with the refinement around the FP64 residual (5e-5); with the FP64
    confirmation (refine_residual = 2) the FP64 residual itself meets 1e-6; a plan without 3xTF32 images
    refuses it with FDA_E_STATE."""
    _need_gpu()
    mesh = inputs.icosphere(14, 0.5)
    k = 100.0
    kw = dict(eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32, alpha=-1j / k)
    S3 = fdbem.Solver(mesh.nodes, mesh.elems, k, m2l_tensor=3, **kw)
    S1 = fdbem.Solver(mesh.nodes, mesh.elems, k, m2l_tensor=1, **kw)
    try:
        x = inputs.complex_gaussian(S3.N, 31)
        xd = torch.from_numpy(x.astype(np.complex64)).to(DEV)
        y3, yt, y1 = torch.empty_like(xd), torch.empty_like(xd), torch.empty_like(xd)
        fdbem.fda_matvec_ex(S3.plan, fdbem.FDA_PREC_FP32, xd, y3)
        fdbem.fda_matvec_ex(S3.plan, fdbem.FDA_PREC_TF32, xd, yt)
        fdbem.fda_matvec_ex(S1.plan, fdbem.FDA_PREC_FP32, xd, y1)
        torch.cuda.synchronize()
        a3, at, a1 = y3.cpu().numpy(), yt.cpu().numpy(), y1.cpu().numpy()
        rows = inputs.sample_rows(S3.N, 256, 7)
        yo = O.matvec_rows(mesh.nodes, mesh.elems, k, x, rows, beta_h=-1j / k)
        for a in (a3, at):
            assert np.linalg.norm(a[rows] - yo) / np.linalg.norm(yo) < 3e-4
        assert np.linalg.norm(at - a1) / np.linalg.norm(a1) < 1e-4
        d = np.linalg.norm(at - a3) / np.linalg.norm(a3)
        assert 1e-7 < d < 5e-4, d
        fdbem.fda_autotune(S3.plan, 1)
        yt2 = torch.empty_like(xd)
        fdbem.fda_matvec_ex(S3.plan, fdbem.FDA_PREC_TF32, xd, yt2)
        xg, yg = xd.clone(), torch.empty_like(xd)
        g = fdbem.fda_matvec_graph_create(S3.plan, fdbem.FDA_PREC_TF32, xg, yg)
        try:
            fdbem.fda_graph_launch(g)
            torch.cuda.synchronize()
            assert (torch.linalg.norm(yg - yt2) / torch.linalg.norm(yt2)).item() < 1e-5
        finally:
            fdbem.fda_graph_destroy(g)
        assert np.linalg.norm(yt2.cpu().numpy() - at) / np.linalg.norm(at) < 2e-5
        b = torch.empty(S3.N, dtype=torch.complex128, device=DEV)
        fdbem.bm_rhs_plane_wave(S3.prob, [0.0, 0.0, 1.0], b)
        u0, u1 = torch.zeros_like(b), torch.zeros_like(b)
        st0 = S3.solve(b, u0, tol=1e-6, restart=100, max_iter=2000, refine=True, inner_tol=1e-3)
        st1 = S3.solve(b, u1, tol=1e-6, restart=100, max_iter=2000, refine=True, inner_tol=1e-3, refine_residual=1)
        assert st0["status"] == fdbem.FDA_OK and st1["status"] == fdbem.FDA_OK and st1["rel_residual"] <= 1e-6
        r = torch.empty_like(b)
        fdbem.fda_matvec_ex(S3.plan, fdbem.FDA_PREC_FP64, u1, r)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(b - r) / torch.linalg.norm(b)).item() < 1e-5
        assert (torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0)).item() < 5e-5
        # refine_residual = 2: the 3xTF32 residual first, then certified with the FP64 operator
        u2 = torch.zeros_like(b)
        st2 = S3.solve(b, u2, tol=1e-6, restart=100, max_iter=2000, refine=True, inner_tol=1e-3, refine_residual=2)
        assert st2["status"] == fdbem.FDA_OK and st2["rel_residual"] <= 1e-6
        fdbem.fda_matvec_ex(S3.plan, fdbem.FDA_PREC_FP64, u2, r)
        torch.cuda.synchronize()
        assert (torch.linalg.norm(b - r) / torch.linalg.norm(b)).item() <= 1.000001e-6
        st = S1.solve(b, torch.zeros_like(b), tol=1e-6, restart=100, max_iter=2000, refine=True, refine_residual=1,
                      raise_on_error=False)
        assert st["status"] == fdbem.FDA_E_STATE and "m2l_tensor = 3" in fdbem.fda_last_error()
        assert fdbem.fda_plan_check(S3.plan) == fdbem.FDA_OK
    finally:
        S1.close()
        S3.close()


def test_near_field_on_tensor_cores_for_wide_batches():
    """The near field of a batch on the tensor cores (near_form = 4: 3xTF32, up to 64 right-hand sides per pass
    over the matrices, off-block corrections by the CSR kernel). Each right-hand side has its own rows of the
    accumulator, so batched columns equal the same plan's single products (1e-6): columns 0, 15, 16 and 19 of
    20 (two TMEM lane quadrants) and 0, 63, 64 and 69 of 70 (a full pass of 64 and a ragged one of 6). Against
    the FP32 FMA stream of the same configuration the product differs by the order of FP32 additions in sums
    with heavy cancellation, in the tensor cores' accumulator and in the FMA lanes (1e-4); both meet the mixed
    bar on 128 oracle rows (3e-4)."""
    _need_gpu()
    mesh = inputs.icosphere(14, 0.5)
    k = 100.0
    kw = dict(eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32, m2l_tensor=1, nrhs_max=70, near_split=1)
    S0 = fdbem.Solver(mesh.nodes, mesh.elems, k, **kw)
    S4 = fdbem.Solver(mesh.nodes, mesh.elems, k, near_form=4, **kw)

    def single(S, col):
        xc = col.contiguous()
        yc = torch.empty_like(xc)
        S.matvec(xc, yc)
        torch.cuda.synchronize()
        return yc

    def rel(a, b):
        return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()

    try:
        rows = inputs.sample_rows(S0.N, 128, 9)
        for nrhs, cols in ((20, (0, 15, 16, 19)), (70, (0, 63, 64, 69))):
            x = inputs.complex_gaussian(S0.N, 50 + nrhs, nrhs=nrhs)
            xd = torch.from_numpy(x.astype(np.complex64)).to(DEV).contiguous()
            y4, y0 = torch.empty_like(xd), torch.empty_like(xd)
            S4.matvec(xd, y4)
            S0.matvec(xd, y0)
            torch.cuda.synchronize()
            diffs = {c: rel(y4[c], single(S4, xd[c])) for c in cols}
            assert max(diffs.values()) < 1e-6, (nrhs, diffs)
            d = rel(y4, y0)
            assert d < 1e-4, (nrhs, d)
            a, b = y4.cpu().numpy(), y0.cpu().numpy()
            for c in cols[::3]:
                yo = _oracle_rows(mesh, k, x[c].astype(np.complex128), rows)
                e4 = np.linalg.norm(a[c][rows] - yo) / np.linalg.norm(yo)
                e0 = np.linalg.norm(b[c][rows] - yo) / np.linalg.norm(yo)
                assert e4 < 3e-4 and e0 < 3e-4, (nrhs, c, e4, e0)
        assert fdbem.fda_plan_check(S4.plan) == fdbem.FDA_OK
    finally:
        S4.close()
        S0.close()


@pytest.mark.parametrize("mode,evict,far", [(0, 1, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0), (1, 1, 0), (0, 0, 1),
                                            (1, 1, 1)])
def test_two_stream_schedule_matches_serial(kd100_variants, mode, evict, far):
    """FP32 products with the far field (S2M, M2M, M2L, L2L) on the plan's own stream beside the near field on
    the caller's stream (two or one near-field CTAs per SM), with the L2 evict-first policy on the near-field
    matrix copies, and with the M2L of each level on its own stream, meet the mixed bar on 256 oracle rows and
    equal the serial product up to the order of the M2L additions; one right-hand side, and a captured graph of
    the product replayed after x is refreshed in place, as well."""
    S, xd, y0, rows, yo = kd100_variants
    fdbem.fda_overlap_force(S.plan, mode, evict, far)
    try:
        yd = torch.empty_like(xd)
        S.matvec(xd, yd)
        torch.cuda.synchronize()
        y = yd.cpu().numpy()
        for r in range(3):
            assert np.linalg.norm(y[r][rows] - yo[r]) / np.linalg.norm(yo[r]) < 3e-4, (mode, r)
            assert np.linalg.norm(y[r] - y0[r]) / np.linalg.norm(y0[r]) < 2e-5, (mode, r)
        x1 = xd[0].contiguous()
        y1 = torch.empty_like(x1)
        S.matvec(x1, y1)
        torch.cuda.synchronize()
        assert np.linalg.norm(y1.cpu().numpy() - y0[0]) / np.linalg.norm(y0[0]) < 2e-5
        xg = torch.zeros_like(xd)
        yg = torch.empty_like(xd)
        g = fdbem.fda_matvec_graph_create(S.plan, fdbem.FDA_PREC_FP32, xg, yg)
        try:
            xg.copy_(xd)
            fdbem.fda_graph_launch(g)
            torch.cuda.synchronize()
            yr = yg.cpu().numpy()
            for r in range(3):
                assert np.linalg.norm(yr[r] - y0[r]) / np.linalg.norm(y0[r]) < 2e-5, (mode, r)
        finally:
            fdbem.fda_graph_destroy(g)
        assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK
    finally:
        fdbem.fda_overlap_force(S.plan, 0, 0, 0)


# ------------------------------------------------------------------ CUDA-graph replay and the autotuner
def test_graph_replay_equals_direct_matvec():
    """A captured product replayed twice (x refreshed in place) equals the direct product of the same x."""
    _need_gpu()
    mesh = inputs.icosphere(6, 0.5)
    S = fdbem.Solver(mesh.nodes, mesh.elems, 20.0, eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     m2l_tensor=1, nrhs_max=4)
    try:
        xd = torch.empty((4, S.N), dtype=torch.complex64, device=DEV)
        yd = torch.empty_like(xd)
        g = fdbem.fda_matvec_graph_create(S.plan, fdbem.FDA_PREC_FP32, xd, yd)
        try:
            assert fdbem.fda_graph_nodes(g) > 10
            for seed in (3, 4):
                x = torch.from_numpy(inputs.complex_gaussian(S.N, seed, nrhs=4).astype(np.complex64)).to(DEV)
                xd.copy_(x)
                fdbem.fda_graph_launch(g)
                torch.cuda.synchronize()
                yr = torch.empty_like(yd)
                fdbem.fda_matvec_ex(S.plan, fdbem.FDA_PREC_FP32, x, yr)
                torch.cuda.synchronize()
                err = (torch.linalg.norm(yd - yr) / torch.linalg.norm(yr)).item()
                assert err < 1e-5, err  # same kernels; only the order of atomic additions differs
        finally:
            fdbem.fda_graph_destroy(g)
    finally:
        S.close()


def test_autotuner_choices_keep_parity():
    """The autotuner times both M2L kernels per (level, stage) and the near-field batch width; the tuned
    plan still meets the mixed-precision bar against the oracle."""
    _need_gpu()
    mesh = inputs.icosphere(8, 0.5)
    k = 20.0
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-5, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     m2l_tensor=1, nrhs_max=16)
    try:
        rep = fdbem.fda_autotune(S.plan, 16)
        assert rep["m2l"] and all(r["ms_fma"] > 0 and r["ms_tensor"] > 0 for r in rep["m2l"])
        assert rep["near_rhs_per_pass"] in (4, 16) and min(rep["near_ms"]) > 0
        x = inputs.complex_gaussian(S.N, 9, nrhs=16)
        xd = torch.from_numpy(x).to(DEV).contiguous()
        yd = torch.empty_like(xd)
        fdbem.fda_matvec_ex(S.plan, fdbem.FDA_PREC_FP32, xd, yd)
        torch.cuda.synchronize()
        rows = inputs.sample_rows(S.N, 100, 7)
        for r in (0, 15):
            yo = _oracle_rows(mesh, k, x[r], rows)
            err = np.linalg.norm(yd[r].cpu().numpy()[rows] - yo) / np.linalg.norm(yo)
            assert err < 3e-4, (r, err)
    finally:
        S.close()


# ------------------------------------------------------------------ radiation data operator B = S + alpha M - alpha/2
def test_radiation_operator_and_pulsating_sphere():
    """Operator B (op = 1) against the oracle's rows on all 1920 rows (FP64: 1e-4), then the pulsating sphere:
    b = B 1 and A u = b solved through the library give the paper's u = a/(1 - ika) within the
    discretisation error of the oracle's own solve (max 5e-3)."""
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    k = 10.0
    N = mesh.n_dof
    SB = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64, op=1)
    SA = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64)
    try:
        q = inputs.complex_gaussian(N, 13)
        qd = torch.from_numpy(q).to(DEV)
        bd = torch.empty_like(qd)
        SB.matvec(qd, bd)
        torch.cuda.synchronize()
        bo = O.radiation_rhs_rows(mesh.nodes, mesh.elems, k, q, np.arange(N))
        assert np.linalg.norm(bd.cpu().numpy() - bo) / np.linalg.norm(bo) < 1e-4
        one = torch.ones(N, dtype=torch.complex128, device=DEV)
        SB.matvec(one, bd)
        u = torch.zeros_like(bd)
        st = SA.solve(bd, u, tol=1e-8, restart=60, max_iter=400)
        assert st["rel_residual"] <= 1e-8
        ue = O.pulsating_sphere(k, 0.5)
        assert np.max(np.abs(u.cpu().numpy() - ue)) < 5e-3 * abs(ue)
    finally:
        SB.close()
        SA.close()


def test_dirichlet_data_recovers_pulsating_velocity():
    """Dirichlet data (f4): with u given, the same Burton-Miller equation is B q = A u (both operators of the
    library). Given the pulsating sphere's u = a/(1 - ika), GMRES on the op = 1 plan returns q = 1."""
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    k = 10.0
    N = mesh.n_dof
    SA = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64)
    SB = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64, op=1)
    try:
        ud = torch.full((N,), complex(O.pulsating_sphere(k, 0.5)), dtype=torch.complex128, device=DEV)
        b = torch.empty_like(ud)
        SA.matvec(ud, b)
        q = torch.zeros_like(b)
        st = SB.solve(b, q, tol=1e-8, restart=60, max_iter=400)
        assert st["rel_residual"] <= 1e-8
        qh = q.cpu().numpy()
        # the library's q satisfies the oracle's own discrete equation B q = A u_D (FDA accuracy) ...
        rows = np.arange(N)
        lhs = O.radiation_rhs_rows(mesh.nodes, mesh.elems, k, qh, rows)
        rhs = O.matvec_rows(mesh.nodes, mesh.elems, k, ud.cpu().numpy(), rows)
        assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-4
        # ... and q = 1 up to the discretisation error of a normal-derivative unknown on 320 elements
        assert np.max(np.abs(qh - 1.0)) < 1.5e-2 and abs(np.mean(qh) - 1.0) < 3e-3
    finally:
        SA.close()
        SB.close()


@pytest.mark.parametrize("form", ["fp64", "mixed"])
def test_robin_data_operator_and_sphere(form):
    """Robin data a u + b q = g (f4; Sec. 2.2, Eq. bm with q = (g - a u)/b eliminated): the plan with op = 2
    applies A + gamma B, gamma = a/b, in one product. Against the oracle's rows of A + gamma B on all 1920 rows
    (FP64 1e-4; mixed form 3e-4); then the sphere with constant g: (A + gamma B) u = (1/b) B g solved through
    the library gives the radiating monopole's u = g / (a + b (1/R - ik)) within the discretisation error of
    320 elements (5e-3 maximum)."""
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    k, R = 10.0, 0.5
    ac, bc = 2.0, 1.0 + 0.5j
    gamma = ac / bc
    N = mesh.n_dof
    kw = dict(precision=fdbem.FDA_PREC_FP32, m2l_tensor=1) if form == "mixed" else {}
    SR = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64, op=2, gamma=gamma, **kw)
    SB = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64, op=1)
    try:
        x = inputs.complex_gaussian(N, 17)
        xd = torch.from_numpy(x).to(DEV)
        yd = torch.empty_like(xd)
        SR.matvec(xd, yd)
        torch.cuda.synchronize()
        yo = O.robin_rows(mesh.nodes, mesh.elems, k, x, np.arange(N), gamma)
        err = np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo)
        assert err < (1e-4 if form == "fp64" else 3e-4), err
        g = torch.ones(N, dtype=torch.complex128, device=DEV)
        b = torch.empty_like(g)
        SB.matvec(g, b)
        b /= bc
        u = torch.zeros_like(b)
        if form == "fp64":
            st = SR.solve(b, u, tol=1e-8, restart=60, max_iter=400)
        else:
            st = SR.solve(b, u, tol=1e-8, restart=60, max_iter=600, refine=True, inner_tol=1e-3)
        assert st["rel_residual"] <= 1e-8
        ue = O.robin_sphere(k, R, ac, bc, 1.0)
        assert np.max(np.abs(u.cpu().numpy() - ue)) < 5e-3 * abs(ue)
    finally:
        SR.close()
        SB.close()


# ------------------------------------------------------------------ failure detection (bounded device waits)
def test_bounded_wait_times_out_and_context_survives():
    """A kernel waits on an mbarrier that nothing completes: its 50 ms bound runs out, it reports the timeout
    and returns; the context keeps working (a product and the plan's error check afterwards)."""
    _need_gpu()
    assert fdbem.fda_wait_selftest(50.0) == 1
    mesh = inputs.icosphere(3, 0.5)
    S = fdbem.Solver(mesh.nodes, mesh.elems, 5.0, eps=1e-4, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                     m2l_tensor=1)
    try:
        x = torch.ones(S.N, dtype=torch.complex128, device=DEV)
        y = torch.empty_like(x)
        S.matvec(x, y)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(y)).all()
        assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK
    finally:
        S.close()


# ------------------------------------------------------------------ full sizes, as the bench runs them
@pytest.mark.parametrize("workload", ["sphere_kd100", "sphere_kd200"])
def test_full_size_sampled_rows(workload):
    """The configurations the bench times (kD = 100: 100,920 DOF; kD = 200: 1,129,080 DOF; eps = 1e-4, 64 points
    per leaf): the autotuned mixed plan (FP32 near field, TF32 tensor-core M2L/M2M/L2L) and its FP64 form
    against the oracle on 256 sampled rows computed one by one (bars 3e-4 and 1e-4)."""
    _need_gpu()
    spec = inputs.WORKLOADS[workload]
    mesh = inputs.make_mesh(spec)
    k = spec["k"]
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=spec["eps"], leaf_max=spec["leaf"],
                     precision=fdbem.FDA_PREC_FP32, m2l_tensor=1)
    try:
        fdbem.fda_autotune(S.plan, 1)
        x = inputs.complex_gaussian(S.N, 20131120)
        xd = torch.from_numpy(x).to(DEV)
        yd = torch.empty_like(xd)
        rows = inputs.sample_rows(S.N, 256, 7)
        yo = _oracle_rows(mesh, k, x, rows)
        for prec, bar in ((fdbem.FDA_PREC_FP32, 3e-4), (fdbem.FDA_PREC_FP64, 1e-4)):
            fdbem.fda_matvec_ex(S.plan, prec, xd, yd)
            torch.cuda.synchronize()
            err = np.linalg.norm(yd.cpu().numpy()[rows] - yo) / np.linalg.norm(yo)
            assert err < bar, (workload, prec, err)
        assert fdbem.fda_plan_check(S.plan) == fdbem.FDA_OK
    finally:
        S.close()


def test_mie_at_kd200():
    """Sec. 5.3 at kD = 200 (eps = 1e-4, 64 points per leaf) on a sphere refined to h ~ lambda/7.8
    (icosphere 130, 2,028,000 DOF, about 105 GB of plan): the mixed refinement solve to a 1e-5 residual is
    within 1e-3 of the Mie series in relative l2 (6.7e-4 measured). The bench's own sphere (h ~ lambda/5.8,
    1,129,080 DOF) sits at 1.6e-3 and the 1,587,000-DOF one at 9.5e-4: the discretisation, not the FDA, sets
    these errors (third order in h). The coupling is alpha = -i/k in the library's normal convention (the
    reading under which the paper's iteration counts hold); the continuous solution does not depend on it."""
    _need_gpu()
    spec = dict(inputs.WORKLOADS["sphere_kd200"], m=130)
    mesh = inputs.make_mesh(spec)
    k = spec["k"]
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=spec["eps"], leaf_max=spec["leaf"],
                     precision=fdbem.FDA_PREC_FP32, m2l_tensor=1, alpha=-1j / k)
    try:
        b = torch.empty(S.N, dtype=torch.complex128, device=DEV)
        fdbem.bm_rhs_plane_wave(S.prob, [0.0, 0.0, 1.0], b)
        x = torch.zeros_like(b)
        st = S.solve(b, x, tol=1e-5, restart=50, max_iter=300, refine=True, inner_tol=1e-3)
        assert st["rel_residual"] <= 1e-5
        xs, _, _ = O.geometry(mesh.nodes, mesh.elems)
        mie = _mie(xs, k, spec["radius"])
        err = np.linalg.norm(x.cpu().numpy() - mie) / np.linalg.norm(mie)
        assert err < 1e-3, err
    finally:
        S.close()
