"""The allocation-free plane-wave right-hand side against the allocating one, through the C ABI.

bm_rhs_plane_wave_noalloc exists for callers that may make CUDA calls but must not allocate device
memory when they build a right-hand side (codes that forbid allocation after start-up, or code that has
handed the rest of the device to another allocator). It keeps the incident directions in a fixed device
array instead of a cudaMalloc'ed buffer. This file is collected last so that a failure here comes after
every other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1311_5202_gb300 import fdbem, inputs  # noqa: E402


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def prob():
    _need_gpu()
    mesh = inputs.icosphere(4, 0.5)
    p = fdbem.bm_problem_create(mesh.nodes, mesh.elems, 10.0)
    yield p, mesh.n_dof
    fdbem.bm_problem_destroy(p)


def _compare(prob, N, dirs, stream=None):
    dev = torch.device("cuda:0")
    nr = dirs.shape[0]
    ref = torch.empty((nr, N), dtype=torch.complex128, device=dev)
    got = torch.full((nr, N), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
    fdbem.bm_rhs_plane_wave(prob, dirs, ref)
    torch.cuda.synchronize()
    fdbem.bm_rhs_plane_wave_noalloc(prob, dirs, got, stream=stream)
    torch.cuda.synchronize()
    a, b = got.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(a))
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


def test_noalloc_rhs_matches_allocating_rhs_on_consecutive_calls(prob):
    p, N = prob
    # two calls in a row with different direction sets: the second overwrites the shared array
    for dirs in (inputs.fibonacci_directions(7) * 3.0, inputs.fibonacci_directions(64)[::-1].copy()):
        _compare(p, N, dirs)


def test_noalloc_rhs_on_a_side_stream_and_at_the_size_limit(prob):
    """A stream other than the default one (the copy into the shared array and the kernel run there), and
    exactly the 1024 directions the fixed array holds."""
    p, N = prob
    side = torch.cuda.Stream()
    _compare(p, N, inputs.fibonacci_directions(5), stream=side)
    _compare(p, N, inputs.fibonacci_directions(1024), stream=side)
    _compare(p, N, inputs.fibonacci_directions(1024)[::-1].copy())


def test_noalloc_rhs_rejects_more_directions_than_the_array_holds(prob):
    p, N = prob
    too_many = np.tile([0.0, 0.0, 1.0], (1025, 1))
    out = torch.zeros((1, N), dtype=torch.complex128, device="cuda:0")
    rc = fdbem.bm_rhs_plane_wave_noalloc(p, too_many, out, raise_on_error=False)
    assert rc == fdbem.FDA_E_INVALID_ARG
    assert "1024" in fdbem.fda_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
