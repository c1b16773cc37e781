"""Synthetic workload definitions: model parameters and their seeded disorder.

Models (paper App. A): the disordered XXZ chain (Eq. xxz), the quantum sun
(Eq. qsun) and a 1D Fermi-Hubbard chain with random on-site potentials.  The
draw order of every random array is fixed here so both sides of every parity
test see identical inputs.  Seeds: realisation r of workload c uses
seed = 1000*c + r.
"""
from dataclasses import dataclass, field
import numpy as np

from .rng import uniform01, normals

XXZ, QSUN, HUBBARD, QREM, QSUN_U1 = 0, 1, 2, 3, 4
PBC, OBC = 0, 1


@dataclass
class XXZParams:
    L: int
    N: int                      # number of up spins (bit = 1)
    J: float = 1.0
    Delta: float = 1.0
    W: float = 0.0
    bc: int = PBC
    seed: int = 0
    h: np.ndarray = field(default=None, repr=False)   # fields h_i, i = 0..L-1
    kind: int = XXZ
    J2: float = 0.0             # next-nearest couplings (Eq. j1j2); 0 = none
    Delta2: float = 1.0
    J3: float = 0.0             # third-neighbour couplings (Eq. j1j2j3); 0 = none
    Delta3: float = 1.0
    phi: float = 0.0            # flux per bond (complex-Hermitian ring); 0 = real


@dataclass
class QSunParams:
    N: int                      # dot spins (top N bits of the state)
    L: int                      # outer spins (bits 0..L-1)
    g0: float = 1.0
    alpha: float = 0.75
    gamma: float = 1.0
    zeta: float = 0.2
    h0: float = 1.0             # field mean
    wh: float = 0.5             # field half-width: h_j ~ U[h0-wh, h0+wh]
    seed: int = 0
    A: np.ndarray = field(default=None, repr=False)       # 2^N x 2^N raw normals
    u_noise: np.ndarray = field(default=None, repr=False)  # u_j - j, U[-zeta, zeta]
    n_of_j: np.ndarray = field(default=None, repr=False)   # dot spin coupled to j
    h: np.ndarray = field(default=None, repr=False)        # fields h_j
    kind: int = QSUN
    M: int = 0                  # U(1) variant: up spins among N + L (the sector)


@dataclass
class HubbardParams:
    L: int
    N_up: int
    N_dn: int
    t: float = 1.0
    U: float = 1.0
    W: float = 0.0
    bc: int = OBC
    seed: int = 0
    mu: np.ndarray = field(default=None, repr=False)     # on-site potentials mu_i
    kind: int = HUBBARD


@dataclass
class QREMParams:
    L: int                      # spins; the full space of 2^L states (row = state)
    Gamma: float = 1.0          # transverse field
    seed: int = 0
    E: np.ndarray = field(default=None, repr=False)      # energies E_alpha, alpha = 0..2^L-1
    kind: int = QREM


def qrem_params(L, Gamma=1.0, seed=0):
    """E_alpha = sqrt(L/2) g_alpha, g_alpha the Box-Muller normals(seed, 2^L) (Eq. qrem: independent
    Gaussian energies with mean 0 and standard deviation sqrt(L/2))."""
    D = 1 << L
    E = np.sqrt(L / 2.0) * normals(seed, D)
    return QREMParams(L=L, Gamma=Gamma, seed=seed, E=E)


def xxz_params(L, N=None, J=1.0, Delta=1.0, W=0.0, bc=PBC, seed=0):
    """h_i = W (2 u_i - 1), u_i = uniform01(seed, i), i = 0..L-1."""
    N = L // 2 if N is None else N
    h = W * (2.0 * uniform01(seed, np.arange(L)) - 1.0)
    return XXZParams(L=L, N=N, J=J, Delta=Delta, W=W, bc=bc, seed=seed, h=h)


def xxz_flux_params(L, phi, N=None, J=1.0, Delta=1.0, W=0.0, bc=PBC, seed=0):
    """The disordered XXZ ring threaded by a flux phi per bond (complex-Hermitian H); fields drawn as
    in xxz_params."""
    p = xxz_params(L, N=N, J=J, Delta=Delta, W=W, bc=bc, seed=seed)
    p.phi = float(phi)
    return p


def j1j2_params(L, N=None, J1=1.0, J2=0.5, Delta1=1.0, Delta2=1.0, J3=0.0, Delta3=1.0, W=1.0, bc=PBC, seed=0):
    """Eq. j1j2 (and Eq. j1j2j3 with J3 != 0); fields drawn as in xxz_params.  The paper's values:
    J1 = 1, J2 = 0.5, Delta1 = Delta2 = 1, W = 1, and J3 = 0.225, Delta3 = 1."""
    p = xxz_params(L, N=N, J=J1, Delta=Delta1, W=W, bc=bc, seed=seed)
    p.J2, p.Delta2, p.J3, p.Delta3 = J2, Delta2, J3, Delta3
    return p


def qsun_params(N=3, L=15, g0=1.0, alpha=0.75, gamma=1.0, zeta=0.2, h0=1.0, wh=0.5, seed=0):
    """Draw order: A (row-major, Box-Muller normals), then u_j noise, n(j), h_j."""
    nd = 1 << N
    A = normals(seed, nd * nd).reshape(nd, nd)
    off = 2 * ((nd * nd + 1) // 2)
    u = uniform01(seed, off + np.arange(3 * L))
    u_noise = zeta * (2.0 * u[:L] - 1.0)
    n_of_j = np.minimum((u[L:2 * L] * N).astype(np.int64), N - 1)
    h = h0 + wh * (2.0 * u[2 * L:] - 1.0)
    return QSunParams(N=N, L=L, g0=g0, alpha=alpha, gamma=gamma, zeta=zeta, h0=h0, wh=wh,
                      seed=seed, A=A, u_noise=u_noise, n_of_j=n_of_j, h=h)


def qsun_u1_params(N=3, L=15, M=None, g0=1.0, alpha=0.75, gamma=1.0, zeta=0.2, h0=1.0, wh=0.5, seed=0):
    """Eq. qsun:U1: the draws of qsun_params (same order), in the sector of M up spins among N + L
    (default (N + L) // 2)."""
    p = qsun_params(N=N, L=L, g0=g0, alpha=alpha, gamma=gamma, zeta=zeta, h0=h0, wh=wh, seed=seed)
    p.kind = QSUN_U1
    p.M = (N + L) // 2 if M is None else M
    return p


def hubbard_params(L, N_up=None, N_dn=None, t=1.0, U=1.0, W=0.0, bc=OBC, seed=0):
    """mu_i = W (2 u_i - 1), u_i = uniform01(seed, i)."""
    N_up = L // 2 if N_up is None else N_up
    N_dn = L // 2 if N_dn is None else N_dn
    mu = W * (2.0 * uniform01(seed, np.arange(L)) - 1.0)
    return HubbardParams(L=L, N_up=N_up, N_dn=N_dn, t=t, U=U, W=W, bc=bc, seed=seed, mu=mu)


def config_seed(config, r):
    return 1000 * config + r


# The five workloads (normalised target eps in [0,1]: lambda = Emin + eps (Emax - Emin)).
CONFIGS = {
    1: dict(name="xxz_L12", model="xxz", L=12, J=1.0, Delta=1.0, W=2.0, nev=20, eps=0.5,
            block=8, precision="f64"),
    2: dict(name="xxz_L20", model="xxz", L=20, J=1.0, Delta=1.0, W=(1.0, 3.0, 5.0), nev=100,
            eps=0.5, block=32, precision=("f64", "f32")),
    3: dict(name="qsun_N3_L15", model="qsun", N=3, L=15, g0=1.0, alpha=0.75, gamma=1.0,
            nev=50, eps=0.5, block=16, precision="f32"),
    4: dict(name="hubbard_L12", model="hubbard", L=12, N_up=6, N_dn=6, t=1.0, U=1.0, W=4.0,
            nev=100, eps=0.5, block=64, precision="f32"),
    5: dict(name="serving_mix", model="xxz", L=(14, 16, 18, 20, 22), W=(0.5, 8.0),
            eps=(0.2, 0.8), nev=(20, 50, 200), requests=2000, precision="f32"),
    # the paper's GPU benchmark model (Eq. qrem), at a size one solve of which takes seconds
    6: dict(name="qrem_L18", model="qrem", L=18, Gamma=1.0, nev=100, eps=0.5, block=32, precision="f32"),
    # the U(1) quantum sun (Eq. qsun:U1) in its half-filled sector, and the J1-J2-J3 chain (Eq. j1j2j3)
    # with the paper's couplings
    7: dict(name="qsun_u1_N3_L15_M9", model="qsun_u1", N=3, L=15, M=9, g0=1.0, alpha=0.75, gamma=1.0,
            nev=50, eps=0.5, block=16, precision="f32"),
    8: dict(name="j1j2j3_L20", model="j1j2", L=20, J2=0.5, J3=0.225, W=1.0, nev=100, eps=0.5, block=32,
            precision="f32"),
}


def serving_stream(n, rate_per_s, Ls=(14, 16, 18, 20, 22), W_range=(0.5, 8.0), eps_range=(0.2, 0.8),
                   nevs=(20, 50, 200), seed=5000):
    """Request stream of the serving workload: n disordered XXZ solves with Poisson arrivals.

    Request k draws five uniforms u = uniform01(seed, 5k + 0..4): L = Ls[floor(u0 len(Ls))],
    W = W_lo + u1 (W_hi - W_lo), eps = eps_lo + u2 (eps_hi - eps_lo),
    nev = nevs[floor(u3 len(nevs))], inter-arrival gap -ln(1 - u4) / rate_per_s.  Its
    fields are those of xxz_params(L, W=W, seed=seed + 1 + k).  Returns a list of dicts
    with keys params, eps, nev, t_arrival (seconds from the stream's start).
    """
    u = uniform01(seed, np.arange(5 * n)).reshape(n, 5)
    out, t = [], 0.0
    for k in range(n):
        L = int(Ls[min(int(u[k, 0] * len(Ls)), len(Ls) - 1)])
        W = W_range[0] + u[k, 1] * (W_range[1] - W_range[0])
        eps = eps_range[0] + u[k, 2] * (eps_range[1] - eps_range[0])
        nev = int(nevs[min(int(u[k, 3] * len(nevs)), len(nevs) - 1)])
        t += -np.log1p(-u[k, 4]) / rate_per_s
        out.append(dict(params=xxz_params(L, W=W, seed=seed + 1 + k), eps=float(eps), nev=nev, t_arrival=t))
    return out
