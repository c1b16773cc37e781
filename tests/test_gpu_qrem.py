"""GPU parity of the QREM model (Eq. qrem) and its structured mapping (custom mappings, Sec. 5.7-5.8).

Bars: the CSR equals the oracle's bit for bit; the structured step (columns generated from bit
flips, one off-diagonal value) equals the CSR step bit for bit in FP64, FP32 and pair-float, for
every block width, and matches the oracle within the FP64 step bound; whole filters and batched
forms (which read the CSR) equal the structured filter bit for bit; a solve matches dense
diagonalisation (eigenvalues within 1e-10 ||H||, residuals <= 1e-9 ||H||).
"""
import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, chebyshev as oc, dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.mark.parametrize("L,Gamma,seed", [(1, 0.5, 1), (6, 1.0, 2), (10, 0.3, 3), (13, 1.7, 4)])
def test_qrem_csr_bitexact(pf, L, Gamma, seed):
    p = pi.qrem_params(L, Gamma=Gamma, seed=seed)
    Hg = pf.Hamiltonian.from_params(p)
    Ho = oh.build(p)
    rp, col, val = (t.cpu().numpy() for t in Hg.csr())
    assert Hg.D == Ho.D == 1 << L and Hg.nnz == Ho.nnz == (L + 1) << L
    assert np.array_equal(rp, Ho.indptr)
    assert np.array_equal(col.astype(np.int64), Ho.indices)
    assert np.array_equal(val, Ho.data)


def _block(shape, seed, dtype):
    x = pi.uniform_pm_half(seed, np.arange(int(np.prod(shape)))).reshape(shape)
    if dtype == "df64":
        hi = x.astype(np.float32)
        lo = (x - hi.astype(np.float64)).astype(np.float32)
        return torch.tensor(np.stack([hi, lo], axis=-1), device="cuda")
    return torch.tensor(x, dtype=torch.float64 if dtype == "f64" else torch.float32, device="cuda")


@pytest.mark.parametrize("L", [10, 13])
@pytest.mark.parametrize("s", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_structured_step_equals_csr(pf, L, s, prec):
    p = pi.qrem_params(L, Gamma=0.9, seed=40 + L)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    D = H.D
    V, B1, B2 = (_block((D, s), 500 + k, prec) for k in range(3))
    outs = {}
    for mapping in ("csr", "structured"):
        H.set_mapping(mapping)
        o = torch.empty_like(V)
        H.clenshaw_step(V, B1, B2, o, 0.0371, 2.0, 1.0)
        o2 = torch.empty_like(V)
        H.clenshaw_step(V, B1, None, o2, -0.25, 1.0, 0.0)
        o3 = torch.empty_like(V)
        H.clenshaw_step(V, None, None, o3, 0.5, 0.0, 0.0)
        outs[mapping] = (o, o2, o3)
    torch.cuda.synchronize()
    for a, b in zip(outs["csr"], outs["structured"]):
        assert torch.equal(a, b)
    if prec == "f64":
        Ec, dE, _, _ = H.rescaled()
        Ht = oc.rescale(oh.build(p), Ec, dE)
        Vn, B1n, B2n = (x.cpu().numpy() for x in (V, B1, B2))
        ref = oc.clenshaw_step(Ht, Vn, B1n, B2n, 0.0371, 2.0)
        S = Ht.scipy().copy()
        S.data = np.abs(S.data)
        bound = 4 * (L + 5) * 2.0 ** -53 * (np.abs(0.0371 * Vn) + 2.0 * (S @ np.abs(B1n)) + np.abs(B2n))
        assert np.all(np.abs(outs["structured"][0].cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_structured_filter_equals_csr_and_batch_forms(pf, prec):
    Hs = []
    items = []
    for j, L in enumerate((9, 11)):
        H = pf.Hamiltonian.from_params(pi.qrem_params(L, Gamma=1.0, seed=60 + j))
        H.spectral_bounds()
        c = pf.filter_coefficients(0.05 * j, [37, 64][j])
        V = _block((H.D, 8), 700 + j, prec)
        items.append((H, V, c))
        Hs.append(H)
    singles = []
    for H, V, c in items:
        W_struct = H.filter_apply(V, c)
        H.set_mapping("csr")
        W_csr = H.filter_apply(V, c)
        H.set_mapping("structured")
        assert torch.equal(W_struct, W_csr)
        singles.append(W_struct)
    for form in ("steps", 1, 4):       # sweeps and persistent kernels read the CSR
        outs = pf.filter_apply_batch(items, form=form)
        for W, Ws in zip(outs, singles):
            assert torch.equal(W, Ws)
    if prec == "f64":
        H, V, c = items[0]
        Ec, dE, _, _ = H.rescaled()
        Ht = oc.rescale(oh.build(pi.qrem_params(9, Gamma=1.0, seed=60)), Ec, dE)
        ref = oc.clenshaw_apply(Ht, V.cpu().numpy(), c)
        err = np.abs(singles[0].cpu().numpy() - ref).max()
        assert err <= (len(c)) * 14 * 2.0 ** -53 * max(1.0, np.abs(ref).max()) * 8


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_qrem_solve_matches_dense(pf, precision):
    p = pi.qrem_params(10, Gamma=1.0, seed=77)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    nev = 20
    K = H.choose_K(0.5, nev)
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + 0.5 * (w[-1] - w[0])
    sel = dense.nearest(w, lam, nev)
    r = H.solve(0.5, nev, K, block=8, precision=precision, target_abs=lam)
    assert r.status == 0
    assert np.max(np.abs(r.evals - w[sel])) <= 1e-10 * hn
    assert np.max(r.resid) <= 1e-9 * hn
    H.set_mapping("csr")
    r2 = H.solve(0.5, nev, K, block=8, precision=precision, target_abs=lam)
    assert np.array_equal(r.evals, r2.evals) and np.array_equal(r.resid, r2.resid)


def test_qrem_server_request(pf):
    sv = pf.Server(block=8, precision="f32")
    p = pi.qrem_params(9, Gamma=0.8, seed=91)
    rid = sv.submit(pf.Model.from_params(p), 0.5, 10)
    r = None
    for _ in range(100000):
        r = sv.take(rid)
        if r is not None:
            break
        sv.step()
    sv.close()
    assert r is not None and r.status == 0
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + 0.5 * (w[-1] - w[0])
    assert np.max(np.abs(np.sort(r.evals) - np.sort(w[dense.nearest(w, lam, 10)]))) <= 1e-10 * hn


@pytest.mark.parametrize("mk", [lambda: pi.hubbard_params(6, 3, 3, U=1.0, W=1.0, bc=pi.PBC, seed=1),
                                lambda: pi.qsun_u1_params(N=2, L=6, M=4, seed=2),
                                lambda: pi.j1j2_params(8, J2=0.5, W=1.0, seed=3)])
def test_structured_mapping_rejected_for_other_models(pf, mk):
    """Models whose off-diagonal elements take more than one value: the periodic Hubbard ring (its
    wrap-around hop carries the Jordan-Wigner sign of the fermions it passes), the U(1) quantum sun
    and the J1-J2 chain keep the CSR."""
    H = pf.Hamiltonian.from_params(mk())
    with pytest.raises(pf.PolfedError):
        H.set_mapping("structured")
    H.set_mapping("csr")


@pytest.mark.parametrize("model", ["xxz", "qsun"])
@pytest.mark.parametrize("L,s,prec", [(12, 8, "f64"), (14, 32, "f32"), (14, 16, "df64"), (16, 32, "f32"),
                                      (9, 1, "f64"), (10, 64, "f32"), (11, 4, "f32")])
def test_csr_column_structured_step_and_filter_equal_csr(pf, model, L, s, prec):
    """Structured mappings that keep the CSR columns: nearest-neighbour XXZ (one off-diagonal value
    (J/2)/dE, per-row diagonal) and the quantum sun (diagonal, dot block, ray couplings) give the
    CSR step's bits, for single steps and whole filters."""
    p = (pi.xxz_params(L, W=2.0, seed=70 + L) if model == "xxz"
         else pi.qsun_params(N=3, L=L - 3, seed=90 + L))
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    V, B1, B2 = (_block((H.D, s), 800 + k, prec) for k in range(3))
    c = pf.filter_coefficients(0.07, 33)
    outs = {}
    for mapping in ("csr", "structured"):
        H.set_mapping(mapping)
        o = torch.empty_like(V)
        H.clenshaw_step(V, B1, B2, o, 0.0219, 2.0, 1.0)
        outs[mapping] = (o, H.filter_apply(V, c))
    torch.cuda.synchronize()
    for a, b in zip(outs["csr"], outs["structured"]):
        assert torch.equal(a, b)
