// (a1) basis enumeration and (a2) CSR Hamiltonian construction on the device.
//
// Basis (paper Sec. 2 intro; App. A.2 binom(L, L/2)): the L-bit integers with N set
// bits in ascending order.  Row r is unranked with the combinatorial number system:
// scanning bit positions p = L-1..0 with k bits still to place, bit p is set iff
// r >= binom(p, k) (then r -= binom(p, k), k -= 1).  The inverse map (rank) is
// sum over the set bits p_1 < p_2 < ... of binom(p_j, j).
//
// Hamiltonians (Eq. xxz, Eq. qsun, open Fermi-Hubbard): one thread per row generates
// the row's terms into a local list, sorts it by column (stable insertion sort) and
// sums repeated columns in generation order.  A count pass, an exclusive scan and a
// fill pass produce the CSR arrays.  Diagonal sums use __dadd_rn/__dmul_rn so that no
// multiply-add is contracted.
#include "common.cuh"
#include <cmath>

namespace pf {

std::atomic<long long> g_kernel_launches{0};
static thread_local char g_cuda_err[256] = {0};
void set_cuda_error(cudaError_t e, const char* where) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
}
const char* last_cuda_error() { return g_cuda_err; }

// ------------------------------------------------------------------ allocator
static pf_alloc_fn g_alloc = nullptr;
static pf_free_fn g_free = nullptr;
static void* g_ctx = nullptr;

void* dev_alloc(size_t bytes, cudaStream_t st) {
  if (bytes == 0) return nullptr;
  if (g_alloc) return g_alloc(g_ctx, bytes, (pf_stream_t)st);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(void* p, cudaStream_t st) {
  if (!p) return;
  if (g_free) {
    g_free(g_ctx, p, (pf_stream_t)st);
    return;
  }
  cudaFreeAsync(p, st);
}

void host_binom(uint64_t* tab) {
  for (int n = 0; n <= 32; ++n)
    for (int k = 0; k <= 32; ++k) {
      uint64_t v;
      if (k > n) v = 0;
      else if (k == 0 || k == n) v = 1;
      else v = tab[(n - 1) * 33 + (k - 1)] + tab[(n - 1) * 33 + k];
      tab[n * 33 + k] = v;
    }
}

// ------------------------------------------------------------------ basis
__device__ __forceinline__ uint32_t unrank_state(uint64_t r, int L, int N, const uint64_t* __restrict__ binom) {
  uint32_t st = 0;
  int k = N;
  for (int p = L - 1; p >= 0 && k > 0; --p) {
    uint64_t c = binom[p * 33 + k];
    if (r >= c) {
      st |= 1u << p;
      r -= c;
      --k;
    }
  }
  return st;
}

__device__ __forceinline__ uint64_t rank_state(uint32_t st, const uint64_t* __restrict__ binom) {
  uint64_t r = 0;
  int j = 1;
  while (st) {
    int p = __ffs(st) - 1;
    r += binom[p * 33 + j];
    ++j;
    st &= st - 1;
  }
  return r;
}

__global__ void unrank_kernel(uint32_t* out, int64_t n, int L, int N, const uint64_t* binom) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = unrank_state((uint64_t)i, L, N, binom);
}

static uint64_t binom_h(int n, int k) {
  // built once; the initialisation of a function-local static is thread-safe
  static const std::vector<uint64_t> tab = [] {
    std::vector<uint64_t> t(33 * 33);
    host_binom(t.data());
    return t;
  }();
  if (n < 0 || k < 0 || n > 32 || k > 32) return 0;
  return tab[n * 33 + k];
}

static pf_status build_basis_impl(const pf_model* m, Basis** out, cudaStream_t st) {
  if (!m || !out) return PF_EINVAL;
  *out = nullptr;
  Basis* b = new Basis();
  b->m = *m;
  b->st = st;
  int L = m->L;
  if (m->kind == PF_MODEL_XXZ) {
    if (L < 1 || L > 32 || m->N < 0 || m->N > L) { delete b; return PF_EINVAL; }
    b->D = (int64_t)binom_h(L, m->N);
  } else if (m->kind == PF_MODEL_HUBBARD) {
    if (L < 2 || L > 31 || m->N_up < 0 || m->N_up > L || m->N_dn < 0 || m->N_dn > L) { delete b; return PF_EINVAL; }
    b->D_up = (int64_t)binom_h(L, m->N_up);
    b->D_dn = (int64_t)binom_h(L, m->N_dn);
    b->D = b->D_up * b->D_dn;
  } else if (m->kind == PF_MODEL_QSUN) {
    if (L < 1 || m->N < 1 || m->N > 5 || m->N + L > 30) { delete b; return PF_EINVAL; }
    b->D = (int64_t)1 << (m->N + L);
  } else if (m->kind == PF_MODEL_QREM) {
    if (L < 1 || L > 30) { delete b; return PF_EINVAL; }
    b->D = (int64_t)1 << L;
  } else if (m->kind == PF_MODEL_QSUN_U1) {
    if (L < 1 || m->N < 1 || m->N > 5 || m->N + L > 32 || m->N_up < 0 || m->N_up > m->N + L) { delete b; return PF_EINVAL; }
    b->D = (int64_t)binom_h(m->N + L, m->N_up);
  } else {
    delete b;
    return PF_EINVAL;
  }
  if (b->D > (int64_t)0x7fffffff) { delete b; return PF_EINVAL; }   // int32 column indices
  uint64_t tab[33 * 33];
  host_binom(tab);
  b->binom = (uint64_t*)dev_alloc(sizeof(tab), st);
  if (!b->binom) { delete b; return PF_ENOMEM; }
  cudaError_t e = cudaMemcpyAsync(b->binom, tab, sizeof(tab), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { set_cuda_error(e, "binom upload"); dev_free(b->binom, st); delete b; return PF_ECUDA; }
  int64_t nst = (m->kind == PF_MODEL_XXZ || m->kind == PF_MODEL_QSUN_U1)
                    ? b->D
                    : (m->kind == PF_MODEL_HUBBARD ? b->D_up + b->D_dn : 0);
  if (nst > 0) {
    b->states = (uint32_t*)dev_alloc(nst * sizeof(uint32_t), st);
    if (!b->states) { dev_free(b->binom, st); delete b; return PF_ENOMEM; }
    if (m->kind == PF_MODEL_XXZ) {
      unrank_kernel<<<(unsigned)ceil_div(b->D, 256), 256, 0, st>>>(b->states, b->D, L, m->N, b->binom);
    } else if (m->kind == PF_MODEL_QSUN_U1) {
      unrank_kernel<<<(unsigned)ceil_div(b->D, 256), 256, 0, st>>>(b->states, b->D, m->N + L, m->N_up, b->binom);
    } else {
      unrank_kernel<<<(unsigned)ceil_div(b->D_up, 256), 256, 0, st>>>(b->states, b->D_up, L, m->N_up, b->binom);
      unrank_kernel<<<(unsigned)ceil_div(b->D_dn, 256), 256, 0, st>>>(b->states + b->D_up, b->D_dn, L, m->N_dn,
                                                                       b->binom);
    }
    PF_COUNT(m->kind == PF_MODEL_HUBBARD ? 2 : 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_cuda_error(e, "unrank_kernel");
      dev_free(b->states, st);
      dev_free(b->binom, st);
      delete b;
      return PF_ECUDA;
    }
  }
  *out = b;
  return PF_OK;
}

// ------------------------------------------------------------------ Hamiltonian
#define PF_MAX_ROW_TERMS 104   // XXZ with three bond ranges at L = 32: 1 + 3 L terms

struct DevModel {
  int kind, L, N, nbonds;
  // XXZ bond ranges q = 0..nranges-1: nbr[q] bonds (i, i + rr[q] mod L) with jdqr = J Delta / 4 and
  // halfJr = J / 2 of that range
  int nranges, nbr[3], rr[3];
  double jdqr[3], halfJr[3];
  int64_t Dd;                 // Hubbard: down-table length
  int flux;                   // XXZ ring with a flux: rows of the real embedding, 2 Dc of them
  int64_t Dc;                 // the sector's dimension
  double fre, fim;            // (J/2) cos(phi), (J/2) sin(phi)
  double jdq, halfJ, negt, U;
  double negG;                // QREM: -Gamma
  const double* E;            // QREM energies [2^L]
  const double* hhalf;        // XXZ/qsun: h_i * 0.5
  const double* mu;           // Hubbard
  const double* hdot;         // qsun: 2^N x 2^N
  const double* coef;         // qsun ray coefficients
  const int32_t* nj;          // qsun dot spin of ray j
  const uint32_t* states;     // XXZ states / Hubbard ups
  const uint32_t* dns;        // Hubbard downs
  const uint64_t* binom;
};

struct RowTerms {
  int32_t c[PF_MAX_ROW_TERMS];
  double v[PF_MAX_ROW_TERMS];
  int n;
  __device__ void push(int64_t col, double val) {
    c[n] = (int32_t)col;
    v[n] = val;
    ++n;
  }
  // stable insertion sort by column, then sum repeated columns in generation order
  __device__ int sort_merge() {
    for (int i = 1; i < n; ++i) {
      int32_t ci = c[i];
      double vi = v[i];
      int j = i - 1;
      while (j >= 0 && c[j] > ci) {
        c[j + 1] = c[j];
        v[j + 1] = v[j];
        --j;
      }
      c[j + 1] = ci;
      v[j + 1] = vi;
    }
    int m = 0;
    for (int i = 0; i < n; ++i) {
      if (m > 0 && c[m - 1] == c[i]) {
        v[m - 1] = __dadd_rn(v[m - 1], v[i]);
      } else {
        c[m] = c[i];
        v[m] = v[i];
        ++m;
      }
    }
    n = m;
    return m;
  }
};

__device__ void gen_row(const DevModel& M, int64_t row, RowTerms& T) {
  T.n = 0;
  const int L = M.L;
  if (M.kind == PF_MODEL_XXZ) {
    // with a flux, row R of the real embedding is part R / Dc of the sector's row R mod Dc
    const int part = (M.flux && row >= M.Dc) ? 1 : 0;
    const int64_t r = row - part * M.Dc;
    uint32_t s = M.states[r];
    double d = 0.0;
    for (int q = 0; q < M.nranges; ++q)
      for (int b = 0; b < M.nbr[q]; ++b) {
        int i = b, j = (b + M.rr[q]) % L;
        bool par = ((s >> i) & 1u) == ((s >> j) & 1u);
        d = __dadd_rn(d, par ? M.jdqr[q] : -M.jdqr[q]);
      }
    for (int i = 0; i < L; ++i) d = __dadd_rn(d, ((s >> i) & 1u) ? M.hhalf[i] : -M.hhalf[i]);
    T.push(row, d);
    if (M.flux) {
      // hop of bond (i, j): A = (J/2) cos(phi); B = +-(J/2) sin(phi), + when spin i is up in s.
      // Part 0 (row r): A at column c, -B at Dc + c; part 1 (row Dc + r): B at c, A at Dc + c.
      for (int b = 0; b < M.nbr[0]; ++b) {
        int i = b, j = (b + 1) % L;
        if (((s >> i) & 1u) != ((s >> j) & 1u)) {
          const int64_t c = (int64_t)rank_state(s ^ ((1u << i) | (1u << j)), M.binom);
          const double B = ((s >> i) & 1u) ? M.fim : -M.fim;
          if (part == 0) {
            if (M.fre != 0.0) T.push(c, M.fre);
            if (B != 0.0) T.push(M.Dc + c, -B);
          } else {
            if (B != 0.0) T.push(c, B);
            if (M.fre != 0.0) T.push(M.Dc + c, M.fre);
          }
        }
      }
      return;
    }
    for (int q = 0; q < M.nranges; ++q)
      for (int b = 0; b < M.nbr[q]; ++b) {
        int i = b, j = (b + M.rr[q]) % L;
        if (((s >> i) & 1u) != ((s >> j) & 1u)) {
          uint32_t t = s ^ ((1u << i) | (1u << j));
          T.push((int64_t)rank_state(t, M.binom), M.halfJr[q]);
        }
      }
  } else if (M.kind == PF_MODEL_QSUN) {
    const int nd = 1 << M.N;
    uint32_t s = (uint32_t)row;
    uint32_t a = s >> L;
    uint32_t outer = s & ((1u << L) - 1u);
    double d = M.hdot[a * nd + a];
    for (int j = 0; j < L; ++j) d = __dadd_rn(d, ((s >> j) & 1u) ? M.hhalf[j] : -M.hhalf[j]);
    T.push(row, d);
    for (int b = 0; b < nd; ++b)
      if ((uint32_t)b != a) T.push((int64_t)(((uint32_t)b << L) | outer), M.hdot[a * nd + b]);
    for (int j = 0; j < L; ++j) {
      uint32_t flip = (1u << (L + M.nj[j])) | (1u << j);
      T.push((int64_t)(s ^ flip), M.coef[j]);
    }
  } else if (M.kind == PF_MODEL_QSUN_U1) {
    const int nd = 1 << M.N;
    const uint32_t s = M.states[row];
    const uint32_t a = s >> L;
    const uint32_t outer = s & ((1u << L) - 1u);
    double d = M.hdot[a * nd + a];
    for (int j = 0; j < L; ++j) d = __dadd_rn(d, ((s >> j) & 1u) ? M.hhalf[j] : -M.hhalf[j]);
    T.push(row, d);
    const int pa = __popc(a);
    for (int q = 0; q < nd; ++q)
      if ((uint32_t)q != a && __popc(q) == pa)
        T.push((int64_t)rank_state(((uint32_t)q << L) | outer, M.binom), M.hdot[a * nd + q]);
    for (int j = 0; j < L; ++j) {
      const int bd = L + M.nj[j];
      if (((s >> bd) & 1u) != ((s >> j) & 1u))
        T.push((int64_t)rank_state(s ^ ((1u << bd) | (1u << j)), M.binom), M.coef[j]);
    }
  } else if (M.kind == PF_MODEL_QREM) {
    T.push(row, M.E[row]);
    for (int i = 0; i < L; ++i) T.push((int64_t)((uint32_t)row ^ (1u << i)), M.negG);
  } else {  // Hubbard
    int64_t iu = row / M.Dd, id = row % M.Dd;
    uint32_t up = M.states[iu], dn = M.dns[id];
    double d = 0.0;
    for (int i = 0; i < L; ++i)
      d = __dadd_rn(d, __dmul_rn(M.U, (double)(((up >> i) & 1u) * ((dn >> i) & 1u))));
    for (int i = 0; i < L; ++i)
      d = __dadd_rn(d, __dmul_rn(M.mu[i], (double)(((up >> i) & 1u) + ((dn >> i) & 1u))));
    T.push(row, d);
    for (int b = 0; b < M.nbonds; ++b) {
      int i = b, j = (b + 1) % L;
      int lo = i < j ? i : j, hi = i < j ? j : i;
      uint32_t mask = (1u << i) | (1u << j);
      uint32_t between = ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
      for (int spin = 0; spin < 2; ++spin) {
        uint32_t occ = spin == 0 ? up : dn;
        if (((occ >> i) & 1u) != ((occ >> j) & 1u)) {
          uint32_t nw = occ ^ mask;
          double sign = (__popc(occ & between) & 1) ? -1.0 : 1.0;
          int64_t c = spin == 0 ? (int64_t)rank_state(nw, M.binom) * M.Dd + id
                                : iu * M.Dd + (int64_t)rank_state(nw, M.binom);
          T.push(c, __dmul_rn(M.negt, sign));
        }
      }
    }
  }
}

__global__ void count_kernel(DevModel M, int64_t D, int64_t* counts) {
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= D) return;
  RowTerms T;
  gen_row(M, row, T);
  counts[row] = T.sort_merge();
}

__global__ void fill_kernel(DevModel M, int64_t D, const int64_t* row_ptr, int32_t* col, double* val) {
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= D) return;
  RowTerms T;
  gen_row(M, row, T);
  int n = T.sort_merge();
  int64_t o = row_ptr[row];
  for (int i = 0; i < n; ++i) {
    col[o + i] = T.c[i];
    val[o + i] = T.v[i];
  }
}

// Exclusive scan of counts[0..n) into out[0..n], out[n] = total.  Three phases with a
// per-block sum array; deterministic.
#define SCAN_BLOCK 1024
__global__ void scan_block_sums(const int64_t* in, int64_t n, int64_t* bsum) {
  __shared__ int64_t sh[32];
  int64_t i = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  v = block_sum<int64_t>(v, sh);
  if (threadIdx.x == 0) bsum[blockIdx.x] = v;
}
__global__ void scan_offsets(int64_t* bsum, int64_t nb) {
  // single thread: nb is D/1024 (small)
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; ++b) {
      int64_t v = bsum[b];
      bsum[b] = acc;
      acc += v;
    }
    bsum[nb] = acc;
  }
}
__global__ void scan_apply(const int64_t* in, int64_t n, const int64_t* boff, int64_t* out) {
  __shared__ int64_t sh[SCAN_BLOCK];
  int64_t i = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
  sh[threadIdx.x] = i < n ? in[i] : 0;
  __syncthreads();
  // Hillis-Steele inclusive scan in shared memory
  for (int o = 1; o < SCAN_BLOCK; o <<= 1) {
    int64_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t incl = sh[threadIdx.x];
  int64_t v = i < n ? in[i] : 0;
  if (i < n) out[i] = boff[blockIdx.x] + incl - v;
  if (i == n - 1) out[n] = boff[blockIdx.x] + incl;
}

static pf_status exclusive_scan(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st) {
  int64_t nb = ceil_div(n, SCAN_BLOCK);
  DevBuf bs;
  PF_TRY(bs.alloc((nb + 1) * sizeof(int64_t), st));
  scan_block_sums<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, n, bs.as<int64_t>());
  scan_offsets<<<1, 32, 0, st>>>(bs.as<int64_t>(), nb);
  scan_apply<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(in, n, bs.as<int64_t>(), out);
  PF_COUNT(2);
  PF_LAUNCH_CHECK("exclusive_scan");
  return PF_OK;
}

// Models whose off-diagonal elements of H share one value, so that a structured mapping can drop
// the value array: QREM (-Gamma, columns from bit flips), the nearest-neighbour XXZ chain (J / 2;
// with L >= 3 no two bonds couple the same pair of states) and the open Hubbard chain (-t: a
// nearest-neighbour hop has no site strictly between its ends, so its Jordan-Wigner sign is +1,
// and an up hop and a down hop never reach the same state).
static bool structured_ok(const Ham* H) {
  if (H->Dc > 0) return false;   // the real embedding of a complex H has two off-diagonal values
  if (H->m.kind == PF_MODEL_QREM || H->m.kind == PF_MODEL_QSUN) return true;
  if (H->m.kind == PF_MODEL_HUBBARD) return H->m.bc != PF_BC_PERIODIC && H->m.L >= 2;
  return H->m.kind == PF_MODEL_XXZ && H->m.J2 == 0.0 && H->m.J3 == 0.0 && H->m.L >= 3;
}

static pf_status build_ham_impl(const Basis* b, const pf_model* m, const pf_params* p, Ham** out, cudaStream_t st) {
  if (!b || !m || !p || !out) return PF_EINVAL;
  *out = nullptr;
  if (m->kind != b->m.kind || m->L != b->m.L || m->N != b->m.N ||
      (m->kind == PF_MODEL_HUBBARD && (m->N_up != b->m.N_up || m->N_dn != b->m.N_dn)) ||
      (m->kind == PF_MODEL_QSUN_U1 && m->N_up != b->m.N_up))
    return PF_EINVAL;
  const int L = m->L;
  DevModel M;
  memset(&M, 0, sizeof(M));
  M.kind = m->kind;
  M.L = L;
  M.N = m->N;
  M.binom = b->binom;
  M.nbonds = (m->bc == PF_BC_PERIODIC) ? L : L - 1;
  // host-side parameter preprocessing (each a single correctly rounded operation)
  std::vector<double> hh, mu, hdot, coef, en;
  std::vector<int32_t> nj;
  if (m->kind == PF_MODEL_XXZ) {
    if (!p->h) return PF_EINVAL;
    M.jdq = (m->J * m->Delta) * 0.25;
    M.halfJ = m->J * 0.5;
    // bond ranges as the oracle lists them: range 1 always, ranges 2 and 3 when their J != 0
    M.nranges = 0;
    const double Jr[3] = {m->J, m->J2, m->J3}, Dr[3] = {m->Delta, m->Delta2, m->Delta3};
    for (int q = 0; q < 3; ++q) {
      if (q > 0 && Jr[q] == 0.0) continue;
      M.rr[M.nranges] = q + 1;
      M.nbr[M.nranges] = (m->bc == PF_BC_PERIODIC) ? L : (L - (q + 1) > 0 ? L - (q + 1) : 0);
      M.jdqr[M.nranges] = (Jr[q] * Dr[q]) * 0.25;
      M.halfJr[M.nranges] = Jr[q] * 0.5;
      ++M.nranges;
    }
    hh.resize(L);
    for (int i = 0; i < L; ++i) hh[i] = p->h[i] * 0.5;
    M.states = b->states;
    if (m->phi != 0.0) {   // complex-Hermitian ring: rows of the real embedding
      if (!std::isfinite(m->phi) || m->J2 != 0.0 || m->J3 != 0.0 || L < 3) return PF_EINVAL;
      M.flux = 1;
      M.Dc = b->D;
      M.fre = M.halfJ * cos(m->phi);
      M.fim = M.halfJ * sin(m->phi);
    }
  } else if (m->kind == PF_MODEL_QSUN) {
    if (!p->h || !p->A || !p->u_noise || !p->n_of_j) return PF_EINVAL;
    M.nbonds = 0;
    int nd = 1 << m->N;
    double c = m->gamma / (sqrt(2.0) * sqrt((double)nd + 1.0));
    hdot.resize(nd * nd);
    for (int a = 0; a < nd; ++a)
      for (int q = 0; q < nd; ++q) hdot[a * nd + q] = (p->A[a * nd + q] + p->A[q * nd + a]) * c;
    hh.resize(L);
    coef.resize(L);
    nj.resize(L);
    for (int j = 0; j < L; ++j) {
      hh[j] = p->h[j] * 0.5;
      double u = (double)j + p->u_noise[j];
      coef[j] = (m->g0 * pow(m->alpha, u)) * 0.25;
      nj[j] = p->n_of_j[j];
      if (nj[j] < 0 || nj[j] >= m->N) return PF_EINVAL;
    }
  } else if (m->kind == PF_MODEL_QSUN_U1) {
    if (!p->h || !p->A || !p->u_noise || !p->n_of_j) return PF_EINVAL;
    M.nbonds = 0;
    const int nd = 1 << m->N, Mup = m->N_up;
    // popcount-conserving part of A + A^T, normalised on the sector: T = sum over a, then b with
    // popcount(b) = popcount(a), of binom(L, M - popcount(a)) (S_ab S_ab); c = gamma / sqrt(T / D)
    double T = 0.0;
    for (int a = 0; a < nd; ++a) {
      const int pa = __builtin_popcount(a);
      const double w = (Mup - pa >= 0 && Mup - pa <= L) ? (double)binom_h(L, Mup - pa) : 0.0;
      for (int q = 0; q < nd; ++q)
        if (__builtin_popcount(q) == pa) {
          const double sv = p->A[a * nd + q] + p->A[q * nd + a];
          T = T + w * (sv * sv);
        }
    }
    if (!(T > 0.0)) return PF_EINVAL;
    const double c = m->gamma / sqrt(T / (double)b->D);
    hdot.assign((size_t)nd * nd, 0.0);
    for (int a = 0; a < nd; ++a)
      for (int q = 0; q < nd; ++q)
        if (__builtin_popcount(q) == __builtin_popcount(a)) hdot[a * nd + q] = (p->A[a * nd + q] + p->A[q * nd + a]) * c;
    hh.resize(L);
    coef.resize(L);
    nj.resize(L);
    for (int j = 0; j < L; ++j) {
      hh[j] = p->h[j] * 0.5;
      double u = (double)j + p->u_noise[j];
      coef[j] = (m->g0 * pow(m->alpha, u)) * 0.5;
      nj[j] = p->n_of_j[j];
      if (nj[j] < 0 || nj[j] >= m->N) return PF_EINVAL;
    }
    M.states = b->states;
  } else if (m->kind == PF_MODEL_QREM) {
    if (!p->E) return PF_EINVAL;
    M.nbonds = 0;
    M.negG = -m->Gamma;
    en.assign(p->E, p->E + b->D);
  } else if (m->kind == PF_MODEL_HUBBARD) {
    if (!p->mu) return PF_EINVAL;
    M.negt = -m->t;
    M.U = m->U;
    mu.assign(p->mu, p->mu + L);
    M.states = b->states;
    M.dns = b->states + b->D_up;
    M.Dd = b->D_dn;
  } else {
    return PF_EINVAL;
  }
  // upload the small arrays in one buffer
  size_t nd_off = 0;
  std::vector<double> blob;
  auto add = [&](const std::vector<double>& v) { size_t o = blob.size(); blob.insert(blob.end(), v.begin(), v.end()); return o; };
  size_t o_hh = add(hh), o_mu = add(mu), o_hd = add(hdot), o_cf = add(coef), o_en = add(en);
  (void)nd_off;
  size_t nblob = blob.size() * sizeof(double) + nj.size() * sizeof(int32_t) + 16;
  DevBuf dblob;
  PF_TRY(dblob.alloc(nblob, st));
  if (!blob.empty()) PF_CUDA(cudaMemcpyAsync(dblob.p, blob.data(), blob.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  int32_t* dnj = (int32_t*)((char*)dblob.p + blob.size() * sizeof(double));
  if (!nj.empty()) PF_CUDA(cudaMemcpyAsync(dnj, nj.data(), nj.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  double* dbl = dblob.as<double>();
  M.hhalf = dbl + o_hh;
  M.mu = dbl + o_mu;
  M.hdot = dbl + o_hd;
  M.coef = dbl + o_cf;
  M.E = dbl + o_en;
  M.nj = dnj;

  Ham* H = new Ham();
  H->m = *m;
  H->D = M.flux ? 2 * b->D : b->D;
  H->Dc = M.flux ? b->D : 0;
  H->st = st;
  const int64_t D = H->D;
  DevBuf counts;
  pf_status s = counts.alloc(D * sizeof(int64_t), st);
  if (s != PF_OK) { delete H; return s; }
  H->row_ptr = (int64_t*)dev_alloc((D + 1) * sizeof(int64_t), st);
  if (!H->row_ptr) { delete H; return PF_ENOMEM; }
  unsigned grid = (unsigned)ceil_div(D, 128);
  count_kernel<<<grid, 128, 0, st>>>(M, D, counts.as<int64_t>());
  PF_COUNT(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_cuda_error(e, "count_kernel"); dev_free(H->row_ptr, st); delete H; return PF_ECUDA; }
  s = exclusive_scan(counts.as<int64_t>(), D, H->row_ptr, st);
  if (s != PF_OK) { dev_free(H->row_ptr, st); delete H; return s; }
  int64_t nnz = 0;
  e = cudaMemcpyAsync(&nnz, H->row_ptr + D, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { set_cuda_error(e, "nnz readback"); dev_free(H->row_ptr, st); delete H; return PF_ECUDA; }
  H->nnz = nnz;
  H->col = (int32_t*)dev_alloc(nnz * sizeof(int32_t), st);
  H->val = (double*)dev_alloc(nnz * sizeof(double), st);
  H->val_t = (double*)dev_alloc(nnz * sizeof(double), st);
  H->val32 = (float*)dev_alloc(nnz * sizeof(float), st);
  H->val_df = (float2*)dev_alloc(nnz * sizeof(float2), st);
  if (!H->col || !H->val || !H->val_t || !H->val32 || !H->val_df) {
    dev_free(H->col, st); dev_free(H->val, st); dev_free(H->val_t, st); dev_free(H->val32, st);
    dev_free(H->val_df, st);
    dev_free(H->row_ptr, st);
    delete H;
    return PF_ENOMEM;
  }
  fill_kernel<<<grid, 128, 0, st>>>(M, D, H->row_ptr, H->col, H->val);
  PF_COUNT(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e, "fill_kernel");
    dev_free(H->col, st); dev_free(H->val, st); dev_free(H->val_t, st); dev_free(H->val32, st);
    dev_free(H->val_df, st);
    dev_free(H->row_ptr, st);
    delete H;
    return PF_ECUDA;
  }
  // structured by default where it is faster: QREM and the XXZ chain; the quantum sun's table
  // lookups cost what the value array saves (34.9 against 34.7 us per FP32 step at N=3, L=15,
  // s=16), so it keeps the CSR unless asked
  H->mapping = (structured_ok(H) && m->kind != PF_MODEL_QSUN) ? PF_MAP_STRUCTURED : PF_MAP_CSR;
  if (m->kind == PF_MODEL_QSUN) {   // the value tables of the structured mapping
    H->qs_hdot = hdot;
    H->qs_coef = coef;
  }
  *out = H;
  return PF_OK;
}

// ------------------------------------------------------------------ rescale and moments
__global__ void rescale_kernel(int64_t D, const int64_t* rp, const int32_t* col, const double* val, double Ec,
                               double dE, double* vt, float* v32, float2* vdf) {
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= D) return;
  for (int64_t j = rp[row]; j < rp[row + 1]; ++j) {
    double x = (col[j] == row) ? (val[j] - Ec) / dE : val[j] / dE;
    vt[j] = x;
    const float hi = (float)x;
    v32[j] = hi;
    vdf[j] = make_float2(hi, (float)(x - (double)hi));   // x - hi is exact in FP64
  }
}

// The diagonal of H~ in the three value forms, copied from the CSR (structured mapping).
__global__ void diag_copy_kernel(int64_t D, const int64_t* rp, const int32_t* col, const double* vt,
                                 const float* v32, const float2* vdf, double* dt, float* d32, float2* ddf) {
  int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= D) return;
  for (int64_t j = rp[row]; j < rp[row + 1]; ++j)
    if (col[j] == row) {
      dt[row] = vt[j];
      d32[row] = v32[j];
      ddf[row] = vdf[j];
    }
}

pf_status set_rescale(Ham* H, double Ec, double dE, cudaStream_t st) {
  if (!(dE > 0.0) || !std::isfinite(Ec) || !std::isfinite(dE)) return PF_EINVAL;
  H->Ec = Ec;
  H->dE = dE;
  rescale_kernel<<<(unsigned)ceil_div(H->D, 256), 256, 0, st>>>(H->D, H->row_ptr, H->col, H->val, Ec, dE, H->val_t,
                                                                 H->val32, H->val_df);
  PF_LAUNCH_CHECK("rescale_kernel");
  if (structured_ok(H)) {
    // structured mapping: every off-diagonal element of H~ is -Gamma / dE (QREM), -t / dE (open
    // Hubbard chain) or (J / 2) / dE (XXZ), the value the rescale kernel computes for each of them;
    // the diagonal is kept per row
    if (!H->diag_t) {
      H->diag_t = (double*)dev_alloc(H->D * sizeof(double), st);
      H->diag32 = (float*)dev_alloc(H->D * sizeof(float), st);
      H->diag_df = (float2*)dev_alloc(H->D * sizeof(float2), st);
      if (!H->diag_t || !H->diag32 || !H->diag_df) return PF_ENOMEM;
    }
    diag_copy_kernel<<<(unsigned)ceil_div(H->D, 256), 256, 0, st>>>(H->D, H->row_ptr, H->col, H->val_t, H->val32,
                                                                    H->val_df, H->diag_t, H->diag32, H->diag_df);
    PF_LAUNCH_CHECK("diag_copy_kernel");
    H->off_t = H->m.kind == PF_MODEL_QREM      ? (-H->m.Gamma) / dE
               : H->m.kind == PF_MODEL_HUBBARD ? (-H->m.t) / dE
                                               : (H->m.J * 0.5) / dE;
    if (H->m.kind == PF_MODEL_QSUN) {
      // the dot block and the ray couplings of H~: off-diagonal elements v / dE, as the rescale
      // kernel computes them, in the three value forms
      const int nt = (int)H->qs_hdot.size(), nc = (int)H->qs_coef.size();
      std::vector<double> t(nt + nc);
      std::vector<float> t32(nt + nc);
      std::vector<float2> tdf(nt + nc);
      for (int k = 0; k < nt + nc; ++k) {
        t[k] = (k < nt ? H->qs_hdot[k] : H->qs_coef[k - nt]) / dE;
        t32[k] = (float)t[k];
        tdf[k] = make_float2(t32[k], (float)(t[k] - (double)t32[k]));
      }
      if (!H->qtab_t) {
        H->qtab_t = (double*)dev_alloc(t.size() * sizeof(double), st);
        H->qtab32 = (float*)dev_alloc(t.size() * sizeof(float), st);
        H->qtab_df = (float2*)dev_alloc(t.size() * sizeof(float2), st);
        if (!H->qtab_t || !H->qtab32 || !H->qtab_df) return PF_ENOMEM;
      }
      H->qtab_n = nt;
      PF_CUDA(cudaMemcpyAsync(H->qtab_t, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      PF_CUDA(cudaMemcpyAsync(H->qtab32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      PF_CUDA(cudaMemcpyAsync(H->qtab_df, tdf.data(), tdf.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
      PF_CUDA(cudaStreamSynchronize(st));   // the host tables are released on return
    }
  }
  H->has_rescale = 1;
  return PF_OK;
}

// partial sums of diag(H~) and of H~_ij^2 per CTA (fixed order), then one CTA sums them.
__global__ void moments_partial(int64_t D, const int64_t* rp, const int32_t* col, const double* vt, double* part) {
  __shared__ double sh[32];
  double tr = 0.0, t2 = 0.0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < D; row += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t j = rp[row]; j < rp[row + 1]; ++j) {
      double x = vt[j];
      if (col[j] == row) tr += x;
      t2 += x * x;
    }
  }
  tr = block_sum(tr, sh);
  t2 = block_sum(t2, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = tr;
    part[2 * blockIdx.x + 1] = t2;
  }
}
__global__ void moments_final(const double* part, int nb, double* out) {
  __shared__ double sh[32];
  double tr = 0.0, t2 = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    tr += part[2 * i];
    t2 += part[2 * i + 1];
  }
  tr = block_sum(tr, sh);
  t2 = block_sum(t2, sh);
  if (threadIdx.x == 0) {
    out[0] = tr;
    out[1] = t2;
  }
}

pf_status ham_moments(Ham* H, double* mu_t, double* G_t, cudaStream_t st) {
  if (!H->has_rescale) return PF_ESTATE;
  const int nb = 592;
  DevBuf part;
  PF_TRY(part.alloc((2 * nb + 2) * sizeof(double), st));
  moments_partial<<<nb, 256, 0, st>>>(H->D, H->row_ptr, H->col, H->val_t, part.as<double>());
  moments_final<<<1, 256, 0, st>>>(part.as<double>(), nb, part.as<double>() + 2 * nb);
  PF_COUNT(1);
  PF_LAUNCH_CHECK("moments");
  double h[2];
  PF_CUDA(cudaMemcpyAsync(h, part.as<double>() + 2 * nb, sizeof(h), cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaStreamSynchronize(st));
  double mu = h[0] / (double)H->D;
  double var = h[1] / (double)H->D - mu * mu;
  *mu_t = mu;
  *G_t = sqrt(var > 0 ? var : 0.0);
  return PF_OK;
}

}  // namespace pf

// ====================================================================== C ABI (basis / H)
using namespace pf;

extern "C" {

pf_status pf_set_allocator(pf_alloc_fn alloc, pf_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return PF_EINVAL;
  g_alloc = alloc;
  g_free = release;
  g_ctx = ctx;
  return PF_OK;
}

const char* pf_last_cuda_error(void) { return g_cuda_err; }

long long pf_kernel_launches(void) { return g_kernel_launches.load(); }

const char* pf_status_str(pf_status s) {
  switch (s) {
    case PF_OK: return "PF_OK";
    case PF_EINVAL: return "PF_EINVAL: invalid argument";
    case PF_ENOMEM: return "PF_ENOMEM: device allocation failed";
    case PF_ENOTCONV: return "PF_ENOTCONV: not converged within the Krylov budget";
    case PF_ETIMEOUT: return "PF_ETIMEOUT: device wait limit reached";
    case PF_ECUDA: return "PF_ECUDA: CUDA error";
    case PF_ESTATE: return "PF_ESTATE: call order violated";
    case PF_EBREAKDOWN: return "PF_EBREAKDOWN: QR breakdown";
  }
  return "unknown pf_status";
}

pf_status pf_build_basis(const pf_model* m, pf_basis** out, pf_stream_t stream) {
  return build_basis_impl(m, reinterpret_cast<Basis**>(out), (cudaStream_t)stream);
}

pf_status pf_basis_info(const pf_basis* bb, int64_t* D, int64_t* D_up, int64_t* D_dn) {
  const Basis* b = reinterpret_cast<const Basis*>(bb);
  if (!b) return PF_EINVAL;
  if (D) *D = b->D;
  if (D_up) *D_up = b->D_up;
  if (D_dn) *D_dn = b->D_dn;
  return PF_OK;
}

pf_status pf_basis_states(const pf_basis* bb, const uint32_t** states) {
  const Basis* b = reinterpret_cast<const Basis*>(bb);
  if (!b || !states) return PF_EINVAL;
  *states = b->states;
  return PF_OK;
}

void pf_free_basis(pf_basis* bb) {
  Basis* b = reinterpret_cast<Basis*>(bb);
  if (!b) return;
  dev_free(b->states, b->st);
  dev_free(b->binom, b->st);
  delete b;
}

pf_status pf_build_hamiltonian(const pf_basis* b, const pf_model* m, const pf_params* p, pf_ham** out,
                               pf_stream_t stream) {
  return build_ham_impl(reinterpret_cast<const Basis*>(b), m, p, reinterpret_cast<Ham**>(out), (cudaStream_t)stream);
}

pf_status pf_ham_info(const pf_ham* hh, int64_t* D, int64_t* nnz, double* norm_est) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H) return PF_EINVAL;
  if (D) *D = H->D;
  if (nnz) *nnz = H->nnz;
  if (norm_est) *norm_est = H->has_bounds ? H->hnorm : 0.0;
  return PF_OK;
}

pf_status pf_ham_csr(const pf_ham* hh, const int64_t** row_ptr, const int32_t** col, const double** val) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H) return PF_EINVAL;
  if (row_ptr) *row_ptr = H->row_ptr;
  if (col) *col = H->col;
  if (val) *val = H->val;
  return PF_OK;
}

void pf_free_ham(pf_ham* hh) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H) return;
  dev_free(H->row_ptr, H->st);
  dev_free(H->col, H->st);
  dev_free(H->val, H->st);
  dev_free(H->val_t, H->st);
  dev_free(H->val32, H->st);
  dev_free(H->val_df, H->st);
  dev_free(H->diag_t, H->st);
  dev_free(H->diag32, H->st);
  dev_free(H->diag_df, H->st);
  dev_free(H->qtab_t, H->st);
  dev_free(H->qtab32, H->st);
  dev_free(H->qtab_df, H->st);
  delete H;
}

pf_status pf_set_rescale(pf_ham* hh, double Ec, double dE, pf_stream_t stream) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H) return PF_EINVAL;
  return set_rescale(H, Ec, dE, (cudaStream_t)stream);
}

pf_status pf_ham_set_mapping(pf_ham* hh, int32_t mapping) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H) return PF_EINVAL;
  if (mapping == PF_MAP_CSR) {
    H->mapping = PF_MAP_CSR;
    return PF_OK;
  }
  if (mapping == PF_MAP_STRUCTURED && structured_ok(H)) {
    H->mapping = PF_MAP_STRUCTURED;
    return PF_OK;
  }
  return PF_EINVAL;
}

pf_status pf_ham_rescaled(const pf_ham* hh, double* Ec, double* dE, const double** val64, const float** val32) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  if (Ec) *Ec = H->Ec;
  if (dE) *dE = H->dE;
  if (val64) *val64 = H->val_t;
  if (val32) *val32 = H->val32;
  return PF_OK;
}

pf_status pf_ham_moments(pf_ham* hh, double* mu_t, double* G_t, pf_stream_t stream) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H || !mu_t || !G_t) return PF_EINVAL;
  return ham_moments(H, mu_t, G_t, (cudaStream_t)stream);
}

}  // extern "C"
