"""Pins of the oracle's Hamiltonians: closed forms, brute force, counts (CPU only)."""
import math
import os
import itertools

import numpy as np
import pytest

import pf_inputs as pi
from oracle import hamiltonian as hm, dense, basis

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_counts():
    out = {}
    for l in open(os.path.join(GOLD, "xxz_offdiag_counts.txt")):
        if not l.startswith("#"):
            L, D, n = map(int, l.split())
            out[L] = (D, n)
    return out


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 14, 16])
def test_xxz_offdiag_count_matches_paper_closed_form(L):
    D, noff = _golden_counts()[L]
    H = hm.xxz_hamiltonian(pi.xxz_params(L, W=1.0, seed=5))
    assert H.D == D
    assert H.nnz - D == noff            # diagonal always stored


def test_xxz_is_symmetric_bitwise_and_rows_sorted():
    H = hm.xxz_hamiltonian(pi.xxz_params(12, W=2.0, seed=1001))
    A = H.scipy()
    assert (A != A.T).nnz == 0
    for r in range(H.D):
        c = H.indices[H.indptr[r]:H.indptr[r + 1]]
        assert np.all(np.diff(c) > 0) and r in c


@pytest.mark.parametrize("L,N", [(4, 2), (6, 3), (8, 4), (10, 5), (12, 6), (8, 3)])
def test_xx_chain_free_fermion_closed_form(L, N):
    H = hm.xxz_hamiltonian(pi.xxz_params(L, N=N, J=1.3, Delta=0.0, W=0.0))
    w, _ = dense.eigh_dense(H)
    assert np.max(np.abs(w - dense.xx_spectrum(L, N, 1.3))) < 1e-12


def test_xxz_wrong_boundary_condition_is_detected():
    # the open chain does NOT have the periodic closed form (guards the bond list)
    H = hm.xxz_hamiltonian(pi.xxz_params(8, J=1.0, Delta=0.0, W=0.0, bc=hm.OBC))
    w, _ = dense.eigh_dense(H)
    assert np.max(np.abs(w - dense.xx_spectrum(8, 4))) > 0.1


def test_heisenberg_ring_L4():
    line = [l for l in open(os.path.join(GOLD, "known_spectra.txt")) if l.startswith("heisenberg_ring_L4_sz0")][0]
    ref = np.array(list(map(float, line.split()[1:])))
    w, _ = dense.eigh_dense(hm.xxz_hamiltonian(pi.xxz_params(4, J=1.0, Delta=1.0, W=0.0)))
    assert np.max(np.abs(w - ref)) < 1e-13


def test_xxz_diagonal_brute_force():
    p = pi.xxz_params(10, J=0.7, Delta=1.9, W=3.0, seed=44)
    H = hm.xxz_hamiltonian(p)
    st = H.states
    dg = H.data[H.diag_mask()]
    for r, s in enumerate(st):
        sz = [((s >> i) & 1) - 0.5 for i in range(p.L)]
        e = sum(p.J * p.Delta * sz[i] * sz[(i + 1) % p.L] for i in range(p.L))
        e += sum(p.h[i] * sz[i] for i in range(p.L))
        assert abs(dg[r] - e) < 1e-13


@pytest.mark.parametrize("L", [6, 8, 12])
def test_xxz_trace_closed_form(L):
    # Tr H / D = -J Delta L / (4 (L-1)) at S^z_tot = 0 with periodic bonds
    p = pi.xxz_params(L, J=1.1, Delta=0.8, W=2.5, seed=9)
    H = hm.xxz_hamiltonian(p)
    tr = H.data[H.diag_mask()].sum() / H.D
    assert abs(tr + p.J * p.Delta * L / (4.0 * (L - 1))) < 1e-12


def test_xxz_L2_duplicates_are_summed():
    H = hm.xxz_hamiltonian(pi.xxz_params(2, J=1.0, Delta=0.0, W=0.0))
    assert H.nnz == 4
    assert np.allclose(H.dense(), [[0, 1.0], [1.0, 0]])


def test_qsun_structure_and_counts():
    p = pi.qsun_params(N=3, L=7, seed=3)
    H = hm.qsun_hamiltonian(p)
    assert H.D == 1 << 10
    assert np.all(np.diff(H.indptr) == (1 << 3) + 7)
    A = H.scipy()
    assert (A != A.T).nnz == 0


def test_qsun_dot_only_spectrum_is_kronecker():
    p = pi.qsun_params(N=2, L=3, g0=0.0, h0=0.0, wh=0.0, seed=11)
    H = hm.qsun_hamiltonian(p)
    w, _ = dense.eigh_dense(H)
    A = p.A
    hd = (A + A.T) / math.sqrt(2.0) * p.gamma / math.sqrt(5.0)
    ref = np.sort(np.repeat(np.linalg.eigvalsh(hd), 1 << 3))
    assert np.max(np.abs(w - ref)) < 1e-13


def test_qsun_fields_and_rays_closed_forms():
    # fields only: E = sum_j h_j (b_j - 1/2)
    p = pi.qsun_params(N=1, L=4, gamma=0.0, g0=0.0, seed=2)
    w, _ = dense.eigh_dense(hm.qsun_hamiltonian(p))
    ref = sorted(sum(p.h[j] * (b[j] - 0.5) for j in range(4)) for b in itertools.product([0, 1], repeat=4) for _ in range(2))
    assert np.max(np.abs(w - np.array(ref))) < 1e-13
    # rays only, one dot spin: all S^x commute, E = sigma_d sum_j c_j sigma_j / 4
    p = pi.qsun_params(N=1, L=3, gamma=0.0, g0=1.3, alpha=0.6, h0=0.0, wh=0.0, seed=8)
    w, _ = dense.eigh_dense(hm.qsun_hamiltonian(p))
    c = [p.g0 * p.alpha ** (j + p.u_noise[j]) for j in range(3)]
    ref = sorted(sd * sum(c[j] * sj[j] for j in range(3)) / 4.0
                 for sd in (-1, 1) for sj in itertools.product([-1, 1], repeat=3))
    assert np.max(np.abs(w - np.array(ref))) < 1e-13


def test_qsun_dot_normalisation_statistical():
    # App. A.2: ||R_dot||^2 = Tr(R_dot^2)/D ~= 1 (expectation exactly 1 for (A+A^T)/sqrt 2 / sqrt(2^N+1))
    vals = []
    for s in range(300):
        p = pi.qsun_params(N=3, L=1, seed=100 + s)
        hd = hm.qsun_dot_matrix(p)
        vals.append(np.sum(hd * hd) / 8.0)
    assert abs(np.mean(vals) - 1.0) < 0.05


@pytest.mark.parametrize("L,Nu,Nd", [(4, 2, 2), (5, 2, 3), (6, 3, 3)])
def test_hubbard_free_fermions_open_chain(L, Nu, Nd):
    H = hm.hubbard_hamiltonian(pi.hubbard_params(L, Nu, Nd, t=0.9, U=0.0, W=0.0))
    w, _ = dense.eigh_dense(H)
    assert np.max(np.abs(w - dense.hubbard_free_spectrum(L, Nu, Nd, 0.9))) < 1e-12


def test_hubbard_dimer_closed_form():
    U = 2.7
    H = hm.hubbard_hamiltonian(pi.hubbard_params(2, 1, 1, t=1.0, U=U, W=0.0))
    w, _ = dense.eigh_dense(H)
    r = math.sqrt(U * U + 16.0)
    assert np.max(np.abs(w - np.sort([0.0, U, (U - r) / 2, (U + r) / 2]))) < 1e-13


def test_hubbard_atomic_limit_and_counts():
    p = pi.hubbard_params(6, 3, 3, t=0.0, U=1.7, W=2.0, seed=7)
    H = hm.hubbard_hamiltonian(p)
    dg = H.data[H.diag_mask()]
    Dd = len(H.dns)
    for r in range(H.D):
        up, dn = H.ups[r // Dd], H.dns[r % Dd]
        e = sum(p.U * ((up >> i) & 1) * ((dn >> i) & 1) + p.mu[i] * (((up >> i) & 1) + ((dn >> i) & 1)) for i in range(6))
        assert abs(dg[r] - e) < 1e-13
    # off-diagonal count, open chain: per species (L-1) * 2 * binom(L-2, N-1) configs x other species
    L, N = 6, 3
    per = (L - 1) * 2 * math.comb(L - 2, N - 1) * math.comb(L, N)
    assert H.nnz - H.D == 2 * per


# ---------------------------------------------------------------- QREM (Eq. qrem)
def _qrem(L, Gamma, E):
    return pi.QREMParams(L=L, Gamma=Gamma, E=np.asarray(E, dtype=np.float64))


@pytest.mark.parametrize("L", [1, 4, 6])
def test_qrem_transverse_field_only_spectrum_closed_form(L):
    # E = 0: H = -Gamma sum_i sigma^x_i, eigenvalues -Gamma (L - 2k) with multiplicity binom(L, k)
    G = 0.7
    w = np.linalg.eigvalsh(hm.build(_qrem(L, G, np.zeros(1 << L))).dense())
    ref = np.sort(np.concatenate([np.full(math.comb(L, k), -G * (L - 2 * k)) for k in range(L + 1)]))
    assert np.max(np.abs(w - ref)) < 1e-12


def test_qrem_two_level_closed_form():
    E0, E1, G = 0.3, -1.1, 0.45
    w = np.linalg.eigvalsh(hm.build(_qrem(1, G, [E0, E1])).dense())
    m, r = 0.5 * (E0 + E1), np.hypot(0.5 * (E0 - E1), G)
    assert np.allclose(w, [m - r, m + r], atol=1e-15)


def test_qrem_structure_diagonal_and_traces():
    L = 7
    p = pi.qrem_params(L, Gamma=0.8, seed=31)
    H = hm.build(p)
    D = 1 << L
    assert H.D == D and H.nnz == D * (L + 1)
    M = H.dense()
    assert np.array_equal(M, M.T)
    assert np.array_equal(np.diag(M), p.E)
    for r in (0, 5, D - 1):
        cols = H.indices[H.indptr[r]:H.indptr[r + 1]]
        assert list(cols) == sorted([r] + [r ^ (1 << i) for i in range(L)])
        off = H.data[H.indptr[r]:H.indptr[r + 1]][cols != r]
        assert np.all(off == -0.8)
    assert abs(np.trace(M) - p.E.sum()) < 1e-12
    assert abs(np.sum(M * M) - (np.sum(p.E ** 2) + L * D * 0.8 ** 2)) < 1e-9


def test_qrem_energies_statistics():
    L = 14
    E = pi.qrem_params(L, seed=7).E
    assert abs(E.mean()) < 4 * np.sqrt(L / 2.0) / np.sqrt(E.size)
    assert abs(E.std() / np.sqrt(L / 2.0) - 1.0) < 0.03


# ---------------------------------------------------------------- J1-J2 (Eq. j1j2) and J1-J2-J3 (Eq. j1j2j3)
@pytest.mark.parametrize("L", [8, 10, 12])
def test_j1j2_majumdar_ghosh_ground_state(L):
    # at J2 = J1/2 (Delta1 = Delta2 = 1, no field, periodic, even L) the two dimer coverings are the
    # exact ground states, with energy -3 J1 L / 8 (Majumdar & Ghosh 1969)
    p = pi.j1j2_params(L, J1=1.0, J2=0.5, W=0.0)
    w = np.linalg.eigvalsh(hm.build(p).dense())
    assert abs(w[0] + 3.0 * L / 8.0) < 1e-10 and abs(w[1] + 3.0 * L / 8.0) < 1e-10
    assert w[2] > w[1] + 1e-3


@pytest.mark.parametrize("L", [7, 9])
def test_range2_only_ring_is_a_relabelled_xxz_ring(L):
    # J1 = 0, odd L: i -> 2i mod L maps the range-2 bonds onto a nearest-neighbour ring
    J2, D2 = 0.8, 0.6
    w2 = np.linalg.eigvalsh(hm.build(pi.j1j2_params(L, N=3, J1=0.0, J2=J2, Delta2=D2, W=0.0)).dense())
    w1 = np.linalg.eigvalsh(hm.build(pi.xxz_params(L, N=3, J=J2, Delta=D2, W=0.0)).dense())
    assert np.max(np.abs(w2 - w1)) < 1e-12


@pytest.mark.parametrize("L,N,J3", [(12, 6, 0.0), (12, 6, 0.225), (11, 4, 0.225)])
def test_j1j2j3_counts_and_trace_closed_forms(L, N, J3):
    p = pi.j1j2_params(L, N=N, J3=J3, W=0.0)
    H = hm.build(p)
    D = math.comb(L, N)
    ranges = [(1, 1.0, 1.0), (2, 0.5, 1.0)] + ([(3, J3, 1.0)] if J3 else [])
    anti = 2 * math.comb(L - 2, N - 1)                     # states antiparallel on a given bond
    par = math.comb(L - 2, N) + math.comb(L - 2, N - 2)
    assert H.D == D and H.nnz == D + len(ranges) * L * anti
    tr = sum(L * (Jr * Dr * 0.25) * (par - anti) for (_, Jr, Dr) in ranges)
    assert abs(np.trace(H.dense()) - tr) < 1e-9
    M = H.dense()
    assert np.array_equal(M, M.T)


def test_j1j2_reduces_to_xxz_when_J2_is_zero():
    a = hm.build(pi.j1j2_params(10, J1=1.3, J2=0.0, Delta1=0.7, W=2.0, seed=5))
    b = hm.build(pi.xxz_params(10, J=1.3, Delta=0.7, W=2.0, seed=5))
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.indices, b.indices)
    assert np.array_equal(a.data, b.data)


# ---------------------------------------------------------------- U(1) quantum sun (Eq. qsun:U1)
def _u1(N, L, M, **kw):
    p = pi.qsun_u1_params(N=N, L=L, M=M, seed=kw.pop("seed", 9))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("N,L,M", [(3, 5, 4), (2, 6, 3), (3, 4, 2)])
def test_qsun_u1_dot_normalisation_and_block_spectrum(N, L, M):
    # g0 = 0, no fields: H = H_dot restricted to the sector.  Tr(H^2)/D = gamma^2 (the numerical
    # normalisation), and the spectrum is that of H_dot's popcount-p blocks, each eigenvalue
    # repeated binom(L, M - p) times.
    p = _u1(N, L, M, g0=0.0, h=np.zeros(L), gamma=1.3)
    Hm = hm.build(p).dense()
    D = math.comb(N + L, M)
    assert Hm.shape == (D, D)
    assert abs(np.trace(Hm @ Hm) / D - 1.3 ** 2) < 1e-12
    hd = hm.qsun_u1_dot_matrix(p)
    pc = basis.popcount(np.arange(1 << N))
    ref = []
    for q in range(N + 1):
        if not 0 <= M - q <= L:
            continue
        blk = np.nonzero(pc == q)[0]
        ev = np.linalg.eigvalsh(hd[np.ix_(blk, blk)])
        ref.extend(np.repeat(ev, math.comb(L, M - q)))
    assert np.max(np.abs(np.linalg.eigvalsh(Hm) - np.sort(ref))) < 1e-12


def test_qsun_u1_single_excitation_star_closed_form():
    # one up spin, no dot term, no fields: the rays hop the excitation between the dot spin and
    # outer spin j with t_j = g0 alpha^u_j / 2, a star graph: eigenvalues +-sqrt(sum t_j^2), 0 (L-1 times)
    N, L = 1, 6
    p = _u1(N, L, 1, gamma=0.0, h=np.zeros(L), n_of_j=np.zeros(L, dtype=np.int64))
    t = 0.5 * p.g0 * np.power(p.alpha, np.arange(L) + p.u_noise)
    w = np.linalg.eigvalsh(hm.build(p).dense())
    r = np.sqrt(np.sum(t * t))
    assert np.allclose(w, np.sort(np.concatenate([[-r, r], np.zeros(L - 1)])), atol=1e-14)


def test_qsun_u1_fields_rays_and_counts():
    N, L, M = 3, 6, 4
    p = _u1(N, L, M, seed=21)
    H = hm.build(p)
    D = math.comb(N + L, M)
    st = H.states
    assert H.D == D and np.array_equal(st, basis.fixed_popcount_states(N + L, M))
    Mx = H.dense()
    assert np.array_equal(Mx, Mx.T)
    # every element conserves the total popcount (automatic in the sector) and the rays carry
    # (g0 alpha^u_j) / 2 between states differing in bits L + n(j) and j only
    coef = (p.g0 * np.power(p.alpha, np.arange(L) + p.u_noise)) * 0.5
    for r in range(D):
        for j0 in range(H.indptr[r], H.indptr[r + 1]):
            c = H.indices[j0]
            x = int(st[r] ^ st[c])
            if c == r or (x >> L) == int(st[r] >> L) ^ int(st[c] >> L) and (x & ((1 << L) - 1)) == 0:
                continue                     # diagonal or a dot-only element
            j = [k for k in range(L) if (x >> k) & 1]
            assert len(j) == 1 and x == (1 << j[0]) | (1 << (L + int(p.n_of_j[j[0]])))
            assert abs(H.data[j0] - coef[j[0]]) <= 4e-16 * abs(coef[j[0]])


# ---------------------------------------------------------------- complex Hermitian: XXZ ring with a flux
def _twisted_xx_levels(L, N, phi, J=1.0):
    """Free fermions of the XX ring with a flux phi per bond: Jordan-Wigner gives one-particle
    energies J cos(k + phi), k = 2 pi (m + shift) / L with shift 1/2 for even N, 0 for odd N
    (the fermions' boundary twist (-1)^(N-1))."""
    shift = 0.5 if N % 2 == 0 else 0.0
    levels = [J * math.cos(2.0 * math.pi * (m + shift) / L + phi) for m in range(L)]
    return np.array(sorted(sum(c) for c in itertools.combinations(levels, N)))


@pytest.mark.parametrize("L,N,phi", [(8, 4, 0.3), (9, 4, 1.1), (10, 5, -0.7), (8, 3, 2.0)])
def test_flux_xx_ring_free_fermion_spectrum(L, N, phi):
    p = pi.xxz_flux_params(L, phi, N=N, Delta=0.0, W=0.0)
    Hc = hm.xxz_flux_hamiltonian(p)
    A = Hc.dense()
    assert np.abs(A - A.conj().T).max() == 0.0
    w = np.linalg.eigvalsh(A)
    assert np.abs(w - _twisted_xx_levels(L, N, phi)).max() < 1e-12
    # a wrong direction of the phase on one bond breaks the closed form
    assert np.abs(np.linalg.eigvalsh(hm.xxz_hamiltonian(pi.xxz_params(L, N=N, Delta=0.0)).dense())
                  - _twisted_xx_levels(L, N, phi)).max() > 1e-3


def test_flux_reduces_to_xxz_and_gauges_away_on_the_open_chain():
    p0 = pi.xxz_params(10, W=2.0, seed=5)
    H0 = hm.xxz_hamiltonian(p0)
    Hz = hm.xxz_flux_hamiltonian(pi.xxz_flux_params(10, 0.0, W=2.0, seed=5))
    assert np.array_equal(Hz.indices, H0.indices) and np.array_equal(Hz.data.real, H0.data)
    assert np.all(Hz.data.imag == 0.0)
    # on the open chain a flux is a gauge transformation: same spectrum as without it
    po = pi.xxz_flux_params(9, 0.9, W=1.5, bc=pi.OBC, seed=6)
    wo = np.linalg.eigvalsh(hm.xxz_flux_hamiltonian(po).dense())
    w0 = np.linalg.eigvalsh(hm.xxz_hamiltonian(pi.xxz_params(9, W=1.5, bc=pi.OBC, seed=6)).dense())
    assert np.abs(wo - w0).max() < 1e-12
    # on the ring it is not: the spectrum moves
    wr = np.linalg.eigvalsh(hm.xxz_flux_hamiltonian(pi.xxz_flux_params(9, 0.9, W=1.5, seed=6)).dense())
    wr0 = np.linalg.eigvalsh(hm.xxz_hamiltonian(pi.xxz_params(9, W=1.5, seed=6)).dense())
    assert np.abs(wr - wr0).max() > 1e-3


def test_real_embedding_doubles_the_spectrum_and_maps_eigenvectors():
    p = pi.xxz_flux_params(10, 0.45, W=2.5, seed=7)
    Hc = hm.xxz_flux_hamiltonian(p)
    M = hm.real_embedding(Hc)
    assert M.D == 2 * Hc.D
    Md = M.dense()
    assert np.array_equal(Md, Md.T)
    w, Z = np.linalg.eigh(Hc.dense())
    wm = np.linalg.eigvalsh(Md)
    assert np.abs(wm - np.repeat(w, 2)).max() < 1e-12 * np.abs(w).max()
    for k in (0, 17, 100):
        z = Z[:, k]
        v = np.concatenate([z.real, z.imag])
        assert np.abs(Md @ v - w[k] * v).max() < 1e-12 * np.abs(w).max()
    assert hm.build(p).D == M.D and np.array_equal(hm.build(p).data, M.data)
