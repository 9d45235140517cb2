"""THC-AO-K (Algorithm 1): the full AO exchange matrix through the C ABI.

K^k = conj(X^k) M^k X^{kT} from thc_build_K against the oracle's
exchange_matrix of its own M, element by element, and E_x against the
oracle's.  Tolerances: FP64 form max|dK| <= 1e-10 max(1, max|K|) and
|dE_x| <= 1e-9 Ha; tensor-core form 1e-6 of max|K| and of |E_x| (the
general mixed bound, as for KC).  Also: K^k is Hermitian for a Hermitian
kernel, and K^k C^k equals the KC of thc_build."""
import numpy as np
import pytest

from oracle import thc_oracle as O
from paper_2304_05505_gb300 import cells

pytestmark = pytest.mark.gpu

CASES = [((3, 2, 2), 20, 4, 46), ((2, 2, 2), 70, 9, 150), ((4, 4, 4), 24, 5, 64), ((6, 6, 6), 12, 3, 40),
         ((1, 1, 1), 5, 2, 7)]


@pytest.fixture(scope="module")
def thc_mod(cuda_required):
    import os
    from paper_2304_05505_gb300 import build_lib, thc
    if not os.path.exists(thc.LIB_PATH):
        build_lib.build()
    thc.load()
    return thc


def _run(thc, r, mesh, precision):
    nk, nb, npt = r["X"].shape
    dims = dict(n1=mesh[0], n2=mesh[1], n3=mesh[2], nbas=nb, nocc=r["C"].shape[2], nisdf=npt)
    eb = thc.ExchangeBuild(dims, precision)
    try:
        eb.set_collocation(r["X"])
        eb.set_kernel(r["V"])
        K, ex = eb.build_K(r["C"])
        eb.sync()
        K = K.cpu().numpy()
        e = float(ex[0])
        KC, ex2 = eb.build(r["C"])        # the same context keeps building THC-oo-K
        eb.sync()
        return K, e, KC.cpu().numpy(), float(ex2[0])
    finally:
        eb.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("mesh,nbas,nocc,nisdf", CASES)
def test_aok_matches_oracle(thc_mod, precision, mesh, nbas, nocc, nisdf):
    r = cells.random_problem(mesh, nbas=nbas, nocc=nocc, nisdf=nisdf, seed=nbas + 3 * nisdf)
    ref = O.build(r["X"], r["C"], r["V"], mesh, keep=True)
    Kref = O.exchange_matrix(r["X"], ref["M"])
    K, ex, KC, ex2 = _run(thc_mod, r, mesh, precision)
    scale = float(np.abs(Kref).max())
    dk = float(np.abs(K - Kref).max())
    if precision == "fp64":
        assert dk <= 1e-10 * max(1.0, scale), dk
        assert abs(ex - ref["Ex"]) <= 1e-9, (ex, ref["Ex"])
    else:
        assert dk <= 1e-6 * scale, (dk, scale)
        assert abs(ex - ref["Ex"]) <= 1e-6 * abs(ref["Ex"]), (ex, ref["Ex"])
    # K is Hermitian for a Hermitian kernel, and K C is the oo build's KC
    herm = float(np.abs(K - np.conj(np.transpose(K, (0, 2, 1)))).max())
    assert herm <= (1e-10 if precision == "fp64" else 2e-6) * scale, herm
    kc = np.einsum("kmn,kni->kmi", K, r["C"])
    tol = 1e-9 if precision == "fp64" else 2e-6
    assert np.abs(kc - KC).max() <= tol * float(np.abs(KC).max())
    assert abs(ex - ex2) <= tol * abs(ex2)


def test_aok_toy_cell(thc_mod):
    """The toy cubic cell (16^3 grid, 2x2x2 k) with the model kernel."""
    p = cells.make_problem("C0")
    ref = O.build(p.X, p.C, p.V, p.cell.mesh, keep=True)
    Kref = O.exchange_matrix(p.X, ref["M"])
    r = dict(X=p.X, C=p.C, V=p.V)
    for precision, tol in (("fp64", 1e-10), ("mixed", 1e-6)):
        K, ex, _, _ = _run(thc_mod, r, p.cell.mesh, precision)
        assert np.abs(K - Kref).max() <= tol * float(np.abs(Kref).max())
        assert abs(ex - ref["Ex"]) <= tol * abs(ref["Ex"])
