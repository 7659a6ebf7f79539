"""The allocation-free plane-wave right-hand side against the allocating one, through the C ABI.

bm_rhs_plane_wave_noalloc exists for callers that cannot allocate device memory when they build a
right-hand side (allocator callbacks, codes that forbid allocation after start-up). It keeps the
incident directions in a fixed device array instead of a cudaMalloc'ed buffer. This file is collected
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1311_5202_gb300 import fdbem, inputs  # noqa: E402


def test_noalloc_rhs_matches_allocating_rhs_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mesh = inputs.icosphere(4, 0.5)
    prob = fdbem.bm_problem_create(mesh.nodes, mesh.elems, 10.0)
    try:
        N = mesh.n_dof
        dev = torch.device("cuda:0")
        # two calls in a row with different direction sets: the second overwrites the shared array
        for dirs in (inputs.fibonacci_directions(7) * 3.0, inputs.fibonacci_directions(64)[::-1].copy()):
            nr = dirs.shape[0]
            ref = torch.empty((nr, N), dtype=torch.complex128, device=dev)
            got = torch.full((nr, N), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
            fdbem.bm_rhs_plane_wave(prob, dirs, ref)
            fdbem.bm_rhs_plane_wave_noalloc(prob, dirs, got)
            torch.cuda.synchronize()
            a, b = got.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
        # more directions than the fixed array holds: a clear error, nothing written
        too_many = np.tile([0.0, 0.0, 1.0], (1025, 1))
        out = torch.zeros((1, N), dtype=torch.complex128, device=dev)
        rc = fdbem.bm_rhs_plane_wave_noalloc(prob, too_many, out, raise_on_error=False)
        assert rc == fdbem.FDA_E_INVALID_ARG
        assert "1024" in fdbem.fda_last_error()
        assert float(out.abs().max()) == 0.0
    finally:
        fdbem.bm_problem_destroy(prob)
