"""Hilbert-space bases (oracle; test infrastructure only).

XXZ (Eq. xxz) conserves total S^z, so the sector with N up spins has dimension
binom(L, N) (App. A.2 quotes binom(L, L/2) for the zero-magnetisation sector).
Convention: bit i of a basis state is 1 when spin i is up.  The sector basis
is the list of L-bit integers with popcount N in ascending order; the row of a
state is its position in that list.

Fermi-Hubbard: a state is a pair (up occupations, down occupations), each an
L-bit integer; row = row_up * D_dn + row_dn with both lists ascending.

Quantum sun (Eq. qsun): no conserved sector; D = 2^(N+L) and the row of a state
is the state itself.  The dot occupies the top N bits.
"""
import numpy as np


def popcount(x):
    x = np.asarray(x, dtype=np.int64)
    c = np.zeros(x.shape, dtype=np.int64)
    for b in range(63):
        c += (x >> b) & 1
    return c


def fixed_popcount_states(L, N):
    """All L-bit integers with exactly N set bits, ascending (brute force)."""
    if N < 0 or N > L:
        return np.zeros(0, dtype=np.int64)
    allx = np.arange(1 << L, dtype=np.int64)
    return allx[popcount(allx) == N]


def row_of(states, targets):
    """Row index of each target state in the ascending ``states`` list."""
    idx = np.searchsorted(states, targets)
    assert np.all(states[np.minimum(idx, len(states) - 1)] == targets)
    return idx


def xxz_basis(L, N):
    return fixed_popcount_states(L, N)


def hubbard_basis(L, N_up, N_dn):
    """Returns (up_states, dn_states); row = i_up * len(dn_states) + i_dn."""
    return fixed_popcount_states(L, N_up), fixed_popcount_states(L, N_dn)


def qsun_basis(N, L):
    return np.arange(1 << (N + L), dtype=np.int64)
