"""The allocation-free entry point against the regular one (collected last on purpose).

shgo_nuclear_attraction_noalloc serves callers that may not allocate device memory: it keeps
everything in the library's static device scratch array.  Its result must equal what
shgo_basis_create + shgo_nuclear_attraction give for the same inputs, call after call, even
though each call reuses (and leaves behind) the previous call's scratch contents."""
import numpy as np
import pytest

from paper_2404_16245_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _regular(shgo, basis, Cd, Zd):
    B = shgo.Basis(basis)
    V = shgo.nuclear_attraction(B, Cd, Zd)
    torch.cuda.synchronize()
    out = V.cpu().numpy()
    B.close()
    return out


def _noalloc(shgo, basis, Cd, Zd):
    n = W.nbf(basis)
    out = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")  # unwritten entries show
    shgo.shgo_nuclear_attraction_noalloc(len(basis["l"]), basis["l"], basis["nprim"], basis["exps"],
                                         basis["coefs"], basis["xyz"], Cd.shape[0], Cd.data_ptr(), Zd.data_ptr(),
                                         out.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_regular_entry_on_consecutive_calls():
    from paper_2404_16245_gb300 import shgo
    big, Cb, Zb = W.config2()   # 32 atoms, l <= 6: 24 MiB of the static scratch
    small, Cs, Zs = W.config1()  # contracted l <= 2
    Cbd, Zbd = torch.tensor(Cb, device="cuda"), torch.tensor(Zb, device="cuda")
    Csd, Zsd = torch.tensor(Cs, device="cuda"), torch.tensor(Zs, device="cuda")
    ref_big = _regular(shgo, big, Cbd, Zbd)
    ref_small = _regular(shgo, small, Csd, Zsd)
    # two calls in a row on the same problem, then a different problem, then the first again
    for basis, Cd, Zd, ref, what in ((big, Cbd, Zbd, ref_big, "first call"), (big, Cbd, Zbd, ref_big, "second call"),
                                     (small, Csd, Zsd, ref_small, "other problem"),
                                     (big, Cbd, Zbd, ref_big, "after other problem")):
        parity.check(_noalloc(shgo, basis, Cd, Zd), ref, what=what)


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    from paper_2404_16245_gb300 import shgo
    # 3000 uncontracted l = 6 shells: 4.5 M pairs x 455 coupling entries, far beyond 64 MiB
    n = 3000
    basis = W.make_basis([6] * n, [1] * n, np.full(n, 1.0), np.ones(n), np.zeros((n, 3)))
    Cd = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    Zd = torch.ones(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_nuclear_attraction_noalloc(n, basis["l"], basis["nprim"], basis["exps"], basis["coefs"],
                                             basis["xyz"], 1, Cd.data_ptr(), Zd.data_ptr(), out.data_ptr())
    assert e.value.status == shgo.ShgoError(1, "").status
    assert "static maximum" in str(e.value)
