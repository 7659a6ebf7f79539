"""Learned leaf-block preconditioner (flexible GMRES): GPU kernels vs the FP64 oracle, and its gain.

The oracle side computes the leaf block solutions from its own dense Nystrom matrix and its own octree
(the leaves are bit-identical to the GPU's), the features, the loss and the gradient by plain
backpropagation in FP64; the GPU runs its FP32 forward/backward kernels. Tolerance 1e-3 relative.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1311_5202_gb300 import fdbem, inputs  # noqa: E402
from paper_1311_5202_gb300 import precond as PC  # noqa: E402

DEV = "cuda:0"


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def c1_precond():
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    k = 10.0
    S = fdbem.Solver(mesh.nodes, mesh.elems, k, eps=1e-6, leaf_max=64, precision=fdbem.FDA_PREC_FP32)
    pc = fdbem.bm_precond_create(S.plan)
    xs, _, _ = O.geometry(mesh.nodes, mesh.elems)
    T = O.tree(xs, 64, k)
    segs = [T["perm"][T["pbeg"][b]:T["pend"][b]] for b in range(len(T["level"])) if T["leaf"][b]]
    A = O.dense_matrix(mesh.nodes, mesh.elems, k)
    yield mesh, S, pc, segs, A
    fdbem.bm_precond_destroy(pc)
    S.close()


def _block_solve(A, segs, r):
    y = np.zeros_like(r)
    for idx in segs:
        y[idx] = np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
    return y


def test_loss_and_gradient_match_oracle(c1_precond):
    mesh, S, pc, segs, A = c1_precond
    H = 16
    net = fdbem.bm_net_create(H, 11)
    try:
        rng = np.random.default_rng(5)
        w = (rng.normal(size=O.net_layout(H)["n"]) * 0.3).astype(np.float32)
        fdbem.bm_net_params(net, w)
        N = S.N
        r = inputs.complex_gaussian(N, 21)
        e = inputs.complex_gaussian(N, 22)
        loss, g = fdbem.bm_precond_train_step(pc, net, torch.from_numpy(r).to(DEV), torch.from_numpy(e).to(DEV),
                                              lr=0.0, want_grad=True)
        y = _block_solve(A, segs, r)
        lo, go = O.net_loss_grad(w.astype(np.float64), H, r, y, e, segs)
        assert abs(loss - lo) < 1e-3 * lo
        assert np.linalg.norm(g - go) < 1e-3 * np.linalg.norm(go)
        # lr = 0 leaves the parameters untouched
        assert np.array_equal(fdbem.bm_net_params(net), w)
    finally:
        fdbem.bm_net_destroy(net)


def test_identity_and_block_modes_match_oracle(c1_precond):
    mesh, S, pc, segs, A = c1_precond
    net = fdbem.bm_net_create(8, 3)
    try:
        N = S.N
        r = inputs.complex_gaussian(N, 31)
        rd = torch.from_numpy(r).to(DEV)
        zd = torch.empty_like(rd)
        PC.net_init(net, "identity")
        fdbem.bm_precond_apply(pc, net, rd, zd)
        z = zd.cpu().numpy()
        assert np.max(np.abs(z - r)) <= 1e-6 * np.max(np.abs(r))  # FP32 round trip
        PC.net_init(net, "block")
        fdbem.bm_precond_apply(pc, net, rd, zd)
        y = _block_solve(A, segs, r)
        assert np.linalg.norm(zd.cpu().numpy() - y) < 1e-4 * np.linalg.norm(y)
    finally:
        fdbem.bm_net_destroy(net)


def test_training_lowers_the_loss(c1_precond):
    mesh, S, pc, segs, A = c1_precond
    net = PC.net_init(fdbem.bm_net_create(16, 5), "identity")
    try:
        R, E = PC.harvest(S, inputs.fibonacci_directions(3), restart=10, cycles=4)
        hist = PC.train(net, [(pc, R, E)], epochs=15, lr=3e-3, batch=4)
        assert hist[-1] < 0.9 * hist[0]
    finally:
        fdbem.bm_net_destroy(net)


def test_learned_preconditioner_cuts_iterations_on_unseen_torus():
    """Trained on random ellipsoids (kD 20-40), judged on a torus (kD 40): flexible GMRES with the network
    needs fewer iterations to the same 1e-5 residual than GMRES without it (coupling -i/k)."""
    _need_gpu()
    train = [(inputs.ellipsoid(8, axes), k) for axes, k in inputs.random_ellipsoid_params(3, seed=1, kd_range=(20, 40))]
    net, info = PC.build_trained(train, alpha_sign=-1, hidden=32, epochs=12, dirs_per_mesh=4)
    try:
        tor = inputs.torus(0.5, 0.2, 48, 20)
        k = 40.0 / 1.4
        S = fdbem.Solver(tor.nodes, tor.elems, k, eps=1e-4, leaf_max=64, precision=fdbem.FDA_PREC_FP32,
                         alpha=-1j / k)
        pc = fdbem.bm_precond_create(S.plan)
        try:
            res = PC.compare(S, pc, net, inputs.fibonacci_directions(2), tol=1e-5, restart=100)
        finally:
            fdbem.bm_precond_destroy(pc)
            S.close()
        for plain, learned in res:
            assert plain["status"] == 0 and learned["status"] == 0
            assert learned["rel_residual"] <= 1e-5
            assert learned["iterations"] < plain["iterations"], (plain["iterations"], learned["iterations"], info)
    finally:
        fdbem.bm_net_destroy(net)
