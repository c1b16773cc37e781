"""CSR Hamiltonians, FP64, built by brute force (oracle; test infrastructure only).

Common conventions (shared with the CUDA builder so that structure AND values
agree bit for bit):
  * Columns in each row are sorted ascending; the diagonal is always stored,
    even when its value is zero.  Repeated (row, col) pairs are summed in the
    order the terms are generated (only XXZ with L = 2 produces any).
  * Diagonal values are accumulated term by term, left to right, starting from
    +0.0, with no fused multiply-add (numpy never contracts a*b+c).

XXZ (Eq. xxz, App. A):  H = J sum_i (S^x_i S^x_{i+1} + S^y_i S^y_{i+1}
                                     + Delta S^z_i S^z_{i+1}) + sum_i h_i S^z_i.
  Bit i = 1 means S^z_i = +1/2.  Bonds (i, i+1) for i = 0..L-2, plus (L-1, 0)
  under periodic boundaries.  An antiparallel bond (i, j) couples the state to
  the one with both spins flipped, with element J/2 (from (S+S- + S-S+)/2).
  Diagonal: for each bond in order, +(J*Delta)*0.25 if parallel else
  -(J*Delta)*0.25; then for i = 0..L-1, +h_i*0.5 if up else -(h_i*0.5).
  J1-J2 (Eq. j1j2) and J1-J2-J3 (Eq. j1j2j3): the same with bonds (i, i+2) of
  coupling J2, Delta2 and (i, i+3) of J3, Delta3 (J1 = J, Delta1 = Delta).  Bonds
  and diagonal terms run range by range (1, then 2, then 3), then the fields; a
  range whose coupling is exactly 0 contributes no bonds.

Quantum sun (Eq. qsun, App. A.2): dot of N spins in the top N bits, outer spin
  j in bit j (j = 0..L-1).  H_dot = gamma R'/sqrt(2^N + 1) with
  R' = (A + A^T)/sqrt(2); element (a, b) is computed as (A_ab + A_ba) * c,
  c = gamma / (sqrt(2) * sqrt(2^N + 1)), and acts on the dot index of states
  that share the outer configuration (the embedding R' (x) I).  Ray j flips
  dot spin n(j) and outer spin j with element (g0 * alpha**u_j) * 0.25
  (S = sigma/2, so S^x S^x has matrix element 1/4), u_j = j + noise_j.
  Diagonal: H_dot[a, a], then for j = 0..L-1, +h_j*0.5 if up else -(h_j*0.5).

Fermi-Hubbard (not in the paper; open chain):
  H = -t sum_{i,sigma} (c+_{i,s} c_{i+1,s} + h.c.) + U sum_i n_i,up n_i,dn
      + sum_i mu_i (n_i,up + n_i,dn).
  Jordan-Wigner order: all up modes, then all down modes, so a hop of one
  species between sites i and j carries (-1)^(occupied sites of that species
  strictly between i and j); element -t times that sign.
  Diagonal: for i = 0..L-1, + U*(n_up_i*n_dn_i); then for i = 0..L-1,
  + mu_i*(n_up_i + n_dn_i) (the occupations as doubles).

U(1) quantum sun (Eq. qsun:U1, App. A.2): the sector of M up spins among the N + L
  bits (dot in the top N), rows in ascending state order as for XXZ.  R' = A + A^T
  with the elements between dot states of different popcount set to zero; H_dot =
  R' c with c = gamma / sqrt(T / D), T = sum over dot states a (ascending), then b
  (ascending) with popcount(b) = popcount(a), of binom(L, M - popcount(a)) *
  (R'_ab * R'_ab), so that Tr(H_dot^2) / D = gamma^2 on the sector.  Ray j flips the
  antiparallel pair (dot spin n(j), outer spin j) with element (g0 * alpha**u_j) * 0.5
  (S^x S^x + S^y S^y).  Diagonal: H_dot[a, a], then the outer fields as above.

XXZ ring with a flux phi per bond (complex Hermitian): each hop carries e^{+-i phi} (see
  xxz_flux_hamiltonian); real_embedding gives the real symmetric [[A, -B], [B, A]] of H = A + iB.

QREM (Eq. qrem, App. A): H = sum_alpha E_alpha |alpha><alpha| - Gamma sum_i sigma^x_i on
  the full space of L spins, row = state.  sigma^x_i flips bit i with element 1, so
  state alpha couples to alpha ^ (1 << i) with element -Gamma for i = 0..L-1.
  Diagonal: E_alpha.
"""
from dataclasses import dataclass, replace as dataclasses_replace
import math

import numpy as np
import scipy.sparse as sp

from . import basis as _basis

PBC, OBC = 0, 1


@dataclass
class CSR:
    D: int
    indptr: np.ndarray    # int64[D+1]
    indices: np.ndarray   # int64[nnz], ascending within each row
    data: np.ndarray      # float64[nnz]

    @property
    def nnz(self):
        return int(self.indptr[-1])

    def scipy(self):
        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.D, self.D))

    def diag_mask(self):
        rows = np.repeat(np.arange(self.D), np.diff(self.indptr))
        return self.indices == rows

    def dense(self):
        return self.scipy().toarray()


def csr_from_terms(D, rows, cols, vals):
    """Sort (row, col) lexicographically (stable) and sum repeated pairs in order."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if len(rows):
        first = np.ones(len(rows), dtype=bool)
        first[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
        if not np.all(first):
            group = np.cumsum(first) - 1
            summed = np.zeros(int(group[-1]) + 1)
            for k in range(len(vals)):          # sequential, generation order
                summed[group[k]] = summed[group[k]] + vals[k]
            rows, cols, vals = rows[first], cols[first], summed
    indptr = np.zeros(D + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=D), out=indptr[1:])
    return CSR(D=D, indptr=indptr, indices=cols, data=vals)


def _bonds(L, bc, r=1):
    """Bonds (i, i + r): i = 0..L-1 (indices mod L) under PBC, i = 0..L-1-r under OBC."""
    nb = L if bc == PBC else max(L - r, 0)
    return [(i, (i + r) % L) for i in range(nb)]


def _coupling_ranges(p):
    """(range, J_r, Delta_r) of Eq. xxz (r = 1), with Eq. j1j2's r = 2 and Eq. j1j2j3's r = 3
    terms when their coupling is nonzero (J_1 = p.J, Delta_1 = p.Delta)."""
    out = [(1, p.J, p.Delta)]
    for r, Jr, Dr in ((2, getattr(p, "J2", 0.0), getattr(p, "Delta2", 1.0)),
                      (3, getattr(p, "J3", 0.0), getattr(p, "Delta3", 1.0))):
        if Jr != 0.0:
            out.append((r, Jr, Dr))
    return out


def xxz_hamiltonian(p):
    """Eq. xxz in the S^z_tot sector with p.N up spins, plus the next-nearest (Eq. j1j2) and
    third-neighbour (Eq. j1j2j3) couplings when p.J2 / p.J3 are nonzero."""
    L = p.L
    states = _basis.xxz_basis(L, p.N)
    D = len(states)
    ranges = [(_bonds(L, p.bc, r), Jr, Dr) for (r, Jr, Dr) in _coupling_ranges(p)]
    d = np.zeros(D)
    for bonds, Jr, Dr in ranges:
        jdq = (Jr * Dr) * 0.25
        for (i, j) in bonds:
            par = ((states >> i) & 1) == ((states >> j) & 1)
            d = d + np.where(par, jdq, -jdq)
    for i in range(L):
        hi = p.h[i] * 0.5
        d = d + np.where(((states >> i) & 1) == 1, hi, -hi)
    rows, cols, vals = [np.arange(D)], [np.arange(D)], [d]
    for bonds, Jr, Dr in ranges:
        half_j = Jr * 0.5
        for (i, j) in bonds:
            anti = ((states >> i) & 1) != ((states >> j) & 1)
            r = np.nonzero(anti)[0]
            t = states[r] ^ ((1 << i) | (1 << j))
            rows.append(r)
            cols.append(_basis.row_of(states, t))
            vals.append(np.full(len(r), half_j))
    H = csr_from_terms(D, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    H.states = states
    return H


def xxz_flux_hamiltonian(p):
    """Eq. xxz on a ring threaded by a flux p.phi per bond: a complex-Hermitian H (Sec. 2 allows
    complex-Hermitian matrices).  The hop of bond (i, j) is (J/2) e^{+i phi} S+_i S-_j + h.c.: the
    element of row state s is (J/2) e^{+i phi} when s has spin i up and j down, (J/2) e^{-i phi} when
    it has i down and j up, with real part (J * 0.5) * cos(phi) and imaginary part +-((J * 0.5) *
    sin(phi)) (the C library's cos and sin).  Diagonal as in xxz_hamiltonian.  complex128 values."""
    Hr = xxz_hamiltonian(dataclasses_replace(p, phi=0.0))
    states = Hr.states
    rows = np.repeat(np.arange(Hr.D), np.diff(Hr.indptr))
    cols = Hr.indices
    half_j = p.J * 0.5
    re, im = half_j * math.cos(p.phi), half_j * math.sin(p.phi)
    data = Hr.data.astype(np.complex128)
    off = rows != cols
    # the one bond joining the row and column states, and which of its ends is up in the row state
    x = states[rows[off]] ^ states[cols[off]]
    lo = np.array([int(v).bit_length() - 1 for v in (x & -x)])       # lower bit of the flipped pair
    hi = np.array([int(v).bit_length() - 1 for v in x])              # higher bit
    wrap = (hi == p.L - 1) & (lo == 0) & (p.L > 2)                   # bond (L-1, 0): i = L-1, j = 0
    i_bit = np.where(wrap, hi, lo)
    up_i = ((states[rows[off]] >> i_bit) & 1) == 1
    data[off] = re + 1j * np.where(up_i, im, -im)
    H = CSR(D=Hr.D, indptr=Hr.indptr, indices=Hr.indices, data=data)
    H.states = states
    return H


def real_embedding(Hc):
    """The real symmetric form [[A, -B], [B, A]] (2D x 2D) of H = A + iB.  Row r < D holds A[r, c] at
    column c and -B[r, c] at D + c; row D + r holds B[r, c] at c and A[r, c] at D + c; entries that are
    exactly zero are not stored, the diagonal always is.  Its spectrum is that of H with every
    eigenvalue twice, and [x; y] is an eigenvector exactly when x + iy is one of H."""
    D = Hc.D
    rows = np.repeat(np.arange(D), np.diff(Hc.indptr))
    cols = Hc.indices
    A, B = Hc.data.real.copy(), Hc.data.imag.copy()
    keepA = (A != 0.0) | (rows == cols)
    keepB = B != 0.0
    r_all = np.concatenate([rows[keepA], rows[keepB], D + rows[keepB], D + rows[keepA]])
    c_all = np.concatenate([cols[keepA], D + cols[keepB], cols[keepB], D + cols[keepA]])
    v_all = np.concatenate([A[keepA], -B[keepB], B[keepB], A[keepA]])
    return csr_from_terms(2 * D, r_all, c_all, v_all)


def qsun_dot_matrix(p):
    """H_dot = gamma (A + A^T)/sqrt(2) / sqrt(2^N + 1) (App. A.2)."""
    nd = 1 << p.N
    c = p.gamma / (np.sqrt(2.0) * np.sqrt(nd + 1.0))
    A = np.asarray(p.A, dtype=np.float64)
    return (A + A.T) * c


def _alpha_pow(alpha, u):
    """alpha**u_j term by term with the C library's pow (math.pow), so that the coupling of each
    ray is one correctly rounded evaluation; numpy's vectorised power may differ in the last bit."""
    return np.array([math.pow(alpha, float(x)) for x in u])


def qsun_ray_coefficients(p):
    """g0 alpha^u_j / 4, u_j = j + noise_j (Eq. qsun; S^x S^x has element 1/4)."""
    u = np.arange(p.L, dtype=np.float64) + p.u_noise
    return (p.g0 * _alpha_pow(p.alpha, u)) * 0.25


def qsun_hamiltonian(p):
    """Eq. qsun on the full 2^(N+L) space."""
    N, L = p.N, p.L
    nd = 1 << N
    D = 1 << (N + L)
    states = _basis.qsun_basis(N, L)
    dot = states >> L
    outer = states & ((1 << L) - 1)
    hd = qsun_dot_matrix(p)
    d = hd[dot, dot].copy()
    for j in range(L):
        hj = p.h[j] * 0.5
        d = d + np.where(((states >> j) & 1) == 1, hj, -hj)
    rows, cols, vals = [states], [states], [d]
    for b in range(nd):
        m = dot != b
        r = states[m]
        rows.append(r)
        cols.append((b << L) | outer[m])
        vals.append(hd[dot[m], b])
    coef = qsun_ray_coefficients(p)
    for j in range(L):
        flip = (1 << (L + int(p.n_of_j[j]))) | (1 << j)
        rows.append(states)
        cols.append(states ^ flip)
        vals.append(np.full(D, coef[j]))
    H = csr_from_terms(D, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    H.states = states
    return H


def qsun_u1_dot_matrix(p):
    """H_dot of Eq. qsun:U1 on the 2^N dot states (zero between different popcounts), normalised
    numerically on the sector of p.M up spins: Tr(H_dot^2) / D = gamma^2."""
    N, L, M = p.N, p.L, p.M
    nd = 1 << N
    A = np.asarray(p.A, dtype=np.float64)
    S = A + A.T
    pc = _basis.popcount(np.arange(nd))
    S = np.where(pc[:, None] == pc[None, :], S, 0.0)
    T = 0.0
    for a in range(nd):
        w = float(math.comb(L, M - int(pc[a]))) if 0 <= M - int(pc[a]) <= L else 0.0
        for b in range(nd):
            if pc[b] == pc[a]:
                T = T + w * (S[a, b] * S[a, b])
    D = math.comb(N + L, M)
    return S * (p.gamma / math.sqrt(T / D))


def qsun_u1_hamiltonian(p):
    """Eq. qsun:U1 in the sector of p.M up spins among N + L."""
    N, L, M = p.N, p.L, p.M
    nd = 1 << N
    states = _basis.fixed_popcount_states(N + L, M)
    D = len(states)
    dot = states >> L
    outer = states & ((1 << L) - 1)
    hd = qsun_u1_dot_matrix(p)
    d = hd[dot, dot].copy()
    for j in range(L):
        hj = p.h[j] * 0.5
        d = d + np.where(((states >> j) & 1) == 1, hj, -hj)
    rows_all = np.arange(D)
    rows, cols, vals = [rows_all], [rows_all], [d]
    pcd = _basis.popcount(dot)
    pcb = _basis.popcount(np.arange(nd))
    for b in range(nd):
        m = (dot != b) & (pcd == pcb[b])
        rows.append(rows_all[m])
        cols.append(_basis.row_of(states, (b << L) | outer[m]))
        vals.append(hd[dot[m], b])
    u = np.arange(L, dtype=np.float64) + p.u_noise
    coef = (p.g0 * _alpha_pow(p.alpha, u)) * 0.5
    for j in range(L):
        bd = L + int(p.n_of_j[j])
        anti = ((states >> bd) & 1) != ((states >> j) & 1)
        r = rows_all[anti]
        rows.append(r)
        cols.append(_basis.row_of(states, states[anti] ^ ((1 << bd) | (1 << j))))
        vals.append(np.full(len(r), coef[j]))
    H = csr_from_terms(D, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    H.states = states
    return H


def _between_mask(i, j):
    lo, hi = min(i, j), max(i, j)
    return ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)


def hubbard_hamiltonian(p):
    L = p.L
    ups, dns = _basis.hubbard_basis(L, p.N_up, p.N_dn)
    Du, Dd = len(ups), len(dns)
    D = Du * Dd
    rows_all = np.arange(D)
    iu, idn = rows_all // Dd, rows_all % Dd
    up, dn = ups[iu], dns[idn]
    d = np.zeros(D)
    for i in range(L):
        d = d + p.U * (((up >> i) & 1) * ((dn >> i) & 1)).astype(np.float64)
    for i in range(L):
        d = d + p.mu[i] * (((up >> i) & 1) + ((dn >> i) & 1)).astype(np.float64)
    rows, cols, vals = [rows_all], [rows_all], [d]
    for (i, j) in _bonds(L, p.bc):
        mask = (1 << i) | (1 << j)
        between = _between_mask(i, j)
        for spin in (0, 1):
            occ = up if spin == 0 else dn
            hop = ((occ >> i) & 1) != ((occ >> j) & 1)
            r = rows_all[hop]
            new = occ[hop] ^ mask
            n_between = _basis.popcount(occ[hop] & between)
            sign = np.where(n_between % 2 == 0, 1.0, -1.0)
            if spin == 0:
                c = _basis.row_of(ups, new) * Dd + idn[hop]
            else:
                c = iu[hop] * Dd + _basis.row_of(dns, new)
            rows.append(r)
            cols.append(c)
            vals.append(-p.t * sign)
    H = csr_from_terms(D, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    H.ups, H.dns = ups, dns
    return H


def qrem_hamiltonian(p):
    """Eq. qrem on the full 2^L space: diagonal E_alpha, single spin flips with -Gamma."""
    L = p.L
    D = 1 << L
    states = np.arange(D, dtype=np.int64)
    rows, cols, vals = [states], [states], [np.asarray(p.E, dtype=np.float64).copy()]
    for i in range(L):
        rows.append(states)
        cols.append(states ^ (1 << i))
        vals.append(np.full(D, -p.Gamma))
    return csr_from_terms(D, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def build(p):
    """Dispatch on the parameter record's model kind (0 XXZ, 1 quantum sun, 2 Hubbard, 3 QREM,
    4 U(1) quantum sun).  An XXZ ring with a flux (p.phi != 0) is complex Hermitian; its real
    embedding (the real symmetric matrix the solver works on) is returned."""
    if p.kind == 0 and getattr(p, "phi", 0.0) != 0.0:
        return real_embedding(xxz_flux_hamiltonian(p))
    return {0: xxz_hamiltonian, 1: qsun_hamiltonian, 2: hubbard_hamiltonian, 3: qrem_hamiltonian,
            4: qsun_u1_hamiltonian}[p.kind](p)
