"""Caller arrays at any 8-byte offset: the right-hand side, the initial guess
and the solution may be views that start 8 bytes past a 16-byte boundary (a
slice of a larger buffer).  Every layout (FP64, mixed one-pass, mixed
streamed) must read and write them element by element as it does aligned
arrays, so the results are bitwise those of aligned arrays, on the device and
through host arrays."""
import numpy as np
import pytest

from paper_2103_07210_gb300 import ftgcr, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _offset_view(a: np.ndarray, dev: str):
    """a copy of a whose data start 8 bytes past a 16-byte boundary."""
    n = a.size
    if dev == "cuda":
        big = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
    else:
        big = torch.zeros(n + 1, dtype=torch.float64).pin_memory()
    v = big[1:].view(a.shape)
    v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    assert v.data_ptr() % 16 == 8
    return v


@pytest.mark.parametrize("nlon,nlat,precision,rounds", [
    (256, 128, "fp64", "auto"),
    (1024, 512, "mixed", "auto"),
    (1024, 64, "mixed", "streamed"),
    (100, 37, "mixed", "auto"),
])
@pytest.mark.parametrize("dev", ["cuda", "host"])
def test_offset_arrays_give_the_aligned_result(nlon, nlat, precision, rounds, dev):
    p = inputs.hill_problem(nlon, nlat, rhs="random", seed=31)
    x0 = 1e-3 * inputs.uniform_pm1(32, p.R.shape)
    with ftgcr.Solver(p.D, p.mu, k=4, tol=1e-10, precision=precision, rounds=rounds) as s:
        R = torch.from_numpy(p.R).cuda()
        xa = torch.from_numpy(x0.copy()).cuda()
        st_a = s.solve(R, xa)
        ref = xa.cpu().numpy()
        Ro = _offset_view(p.R, dev)
        xo = _offset_view(x0, dev)
        st_o = s.solve(Ro, xo)
        got = xo.cpu().numpy()
    assert st_a == ftgcr.OK and st_o == ftgcr.OK
    assert np.array_equal(got, ref)
