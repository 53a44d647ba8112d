// AIRG setup on the GPU: every step of Section "AIRG" (setup steps 1-11) as CUDA kernels.
//
//   step 1  CF splitting ........ strength (eq. soc), PMISR (Algorithm 1), DDC (Algorithm 2)
//   step 2  extraction .......... stable F/C renumbering by prefix sums, A_ff / A_fc / A_cf
//   steps 3-6 polynomial fit .... Box-Muller rhs, power basis by SpMV, Householder TSQR, Givens LSQ
//   steps 7-8 approximate inverse first-order fixed-sparsity powers, assembled Ainv
//   step 9  restrictor .......... Z = -A_cf Ainv with the relative row-wise inf-norm drop
//   step 10 prolongator ......... classical one-point map (weight 1)
//   step 11 coarse matrix ....... A_c = R (A P) with drop, diagonal kept
//
// Integer decisions (strength flags, PMISR, DDC, patterns, drops) and the product values are
// computed in a fixed arithmetic order (ascending index, explicit fma) so that, given the same
// input matrix and coefficients, they reproduce the plain definitions bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "airg_common.cuh"

namespace airg {

// ------------------------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  Output c of a
// stream keyed by K is mix(K + (c+1) * gamma); keys are derived from (seed, level, stream).
// ------------------------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// stream 0: PMISR tie-break weights, stream 1: Box-Muller right-hand side
__host__ __device__ __forceinline__ uint64_t sm64_key(uint64_t seed, int level, int stream) {
  return sm64_mix(seed + kGamma * (uint64_t)(1 + 2 * level + stream));
}
__device__ __forceinline__ double sm64_unif(uint64_t key, uint64_t c) {
  return (double)(sm64_mix(key + kGamma * (c + 1)) >> 11) * (1.0 / 9007199254740992.0);
}

#define GRID(n) grid_for((n), 256), 256, 0, s

// ------------------------------------------------------------------------------------------
// Input validation
// ------------------------------------------------------------------------------------------
__global__ void k_validate(int n, int nnz, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ v, int* flags) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    int b = rp[i], e = rp[i + 1];
    if (b < 0 || e < b || e > nnz) { atomicOr(flags, 1); continue; }
    bool diag = false;
    for (int k = b; k < e; ++k) {
      int j = ci[k];
      if (j < 0 || j >= n || (k > b && j <= ci[k - 1])) atomicOr(flags, 1);
      if (j == i) diag = (v[k] != 0.0);
    }
    if (!diag) atomicOr(flags, 2);
  }
}

int validate_csr(const DCsr& A, Arena& tmp, cudaStream_t s) {
  int* flags;
  AIRG_TRY(tmp.alloc(&flags, 1));
  CU_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  int ends[2] = {0, 0};
  CU_TRY(cudaMemcpyAsync(&ends[0], A.rp, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaMemcpyAsync(&ends[1], A.rp + A.nrows, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (A.nrows > 0) airg::note_launch(), k_validate<<<GRID(A.nrows)>>>(A.nrows, A.nnz, A.rp, A.ci, A.v, flags);
  KERNEL_CHECK();
  int h = 0;
  CU_TRY(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != A.nnz || (h & 1)) return AIRG_ERR_CSR;
  if (h & 2) return AIRG_ERR_ZERO_DIAG;
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Step 1a: strength of connection, eq. soc with absolute values.  strong(i,j) iff j != i,
// a_ij != 0 and |a_ij| >= alpha * max_{k != i} |a_ik|; a row with zero off-diagonal maximum has
// no strong entry.  nS[i] = |S_i|.
// ------------------------------------------------------------------------------------------
// The bit pattern of a non-negative double, read as a signed 64-bit integer, orders exactly like the
// value; comparisons of magnitudes therefore run on the integer pipe (FP64 issue is scarce on
// sm_103a) with results identical to the FP64 comparisons.
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }

// Row kernels walk their entries in batches of kGB: the batch's column loads, then its gathers of
// per-column state, are issued together (two memory latencies per batch instead of two per entry).
constexpr int kGB = 4;

__global__ void k_strength(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                           double alpha, uint8_t* __restrict__ strong, int* __restrict__ nS) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = rp[i], e = rp[i + 1];
    long long mx = 0;
    for (int k = b; k < e; ++k)
      if (ci[k] != i) mx = max(mx, abs_bits(v[k]));
    // alpha * max in FP64 (one multiply per row), then |a_ij| >= threshold on the bit patterns
    const long long thr = abs_bits(alpha * __longlong_as_double(mx));
    int cnt = 0;
    for (int k = b; k < e; ++k) {
      const long long a = abs_bits(v[k]);
      const bool st = (mx != 0) && (ci[k] != i) && (a != 0) && (a >= thr);
      strong[k] = st;
      cnt += st;
    }
    nS[i] = cnt;
  }
}

// |S_i^T| and the transpose adjacency (order within a row is irrelevant: it is used as a set)
__global__ void k_strong_T_count(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const uint8_t* __restrict__ strong, int* nST) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (strong[k]) atomicAdd(nST + ci[k], 1);
}
__global__ void k_strong_T_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const uint8_t* __restrict__ strong, const int* __restrict__ rpT, int* cursor,
                                int* __restrict__ colT) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (strong[k]) {
        int j = ci[k];
        int p = atomicAdd(cursor + j, 1);
        colT[rpT[j] + p] = (int)i;
      }
}

// ------------------------------------------------------------------------------------------
// Step 1b: PMISR, Algorithm 1.  w_i = |S_i| + |S_i^T| + r_i; {w < 1} (isolated nodes) start as F.
// Each round: D = unassigned nodes whose (w, index) is smaller than that of every unassigned
// neighbour in S_i u S_i^T (state frozen at the round start); D -> F, unassigned neighbours of D
// -> C.  After n_loops^max rounds the remaining nodes become C.
// ------------------------------------------------------------------------------------------
__global__ void k_pmisr_init(int n, const int* __restrict__ nS, const int* __restrict__ nST, uint64_t key,
                             double* __restrict__ w, int8_t* __restrict__ cf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int deg = nS[i] + nST[i];
    const double wi = (double)deg + sm64_unif(key, (uint64_t)i);
    w[i] = wi;
    cf[i] = (wi < 1.0) ? (int8_t)kF : (int8_t)0;
  }
}

// (w_i, i) < (w_j, j); weights are non-negative, so their bit patterns compare as integers
__device__ __forceinline__ bool pmisr_less(long long wi, int i, long long wj, int j) {
  return wi < wj || (wi == wj && i < j);
}

__global__ void k_pmisr_select(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                               const uint8_t* __restrict__ strong, const int* __restrict__ rpT,
                               const int* __restrict__ colT, const double* __restrict__ w,
                               const int8_t* __restrict__ cf, uint8_t* __restrict__ D) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    uint8_t isD = 0;
    if (cf[i] == 0) {
      const long long wi = __double_as_longlong(w[i]);
      bool mn = true;
      const int e = rp[i + 1];
      for (int k0 = rp[i]; k0 < e && mn; k0 += kGB) {
        int j[kGB];
        int8_t c[kGB];
        long long wj[kGB];
#pragma unroll
        for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < e && strong[k0 + t]) ? ci[k0 + t] : -1;
#pragma unroll
        for (int t = 0; t < kGB; ++t) {
          c[t] = (j[t] >= 0) ? cf[j[t]] : (int8_t)1;
          wj[t] = (j[t] >= 0) ? __double_as_longlong(w[j[t]]) : 0;
        }
#pragma unroll
        for (int t = 0; t < kGB; ++t)
          if (c[t] == 0 && !pmisr_less(wi, i, wj[t], j[t])) mn = false;
      }
      const int eT = rpT[i + 1];
      for (int k0 = rpT[i]; k0 < eT && mn; k0 += kGB) {
        int j[kGB];
        int8_t c[kGB];
        long long wj[kGB];
#pragma unroll
        for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < eT) ? colT[k0 + t] : -1;
#pragma unroll
        for (int t = 0; t < kGB; ++t) {
          c[t] = (j[t] >= 0) ? cf[j[t]] : (int8_t)1;
          wj[t] = (j[t] >= 0) ? __double_as_longlong(w[j[t]]) : 0;
        }
#pragma unroll
        for (int t = 0; t < kGB; ++t)
          if (c[t] == 0 && !pmisr_less(wi, i, wj[t], j[t])) mn = false;
      }
      isD = mn;
    }
    D[i] = isD;
  }
}

__global__ void k_pmisr_apply(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const uint8_t* __restrict__ strong, const int* __restrict__ rpT,
                              const int* __restrict__ colT, const uint8_t* __restrict__ D, int8_t* __restrict__ cf,
                              int* n_unassigned) {
  int left = 0;
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    if (cf[i] != 0) continue;
    if (D[i]) { cf[i] = kF; continue; }
    bool nbD = false;
    const int e = rp[i + 1];
    for (int k0 = rp[i]; k0 < e && !nbD; k0 += kGB) {
      int j[kGB];
#pragma unroll
      for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < e && strong[k0 + t]) ? ci[k0 + t] : -1;
#pragma unroll
      for (int t = 0; t < kGB; ++t)
        if (j[t] >= 0 && D[j[t]]) nbD = true;
    }
    const int eT = rpT[i + 1];
    for (int k0 = rpT[i]; k0 < eT && !nbD; k0 += kGB) {
      int j[kGB];
#pragma unroll
      for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < eT) ? colT[k0 + t] : -1;
#pragma unroll
      for (int t = 0; t < kGB; ++t)
        if (j[t] >= 0 && D[j[t]]) nbD = true;
    }
    if (nbD) cf[i] = kC;
    else left++;
  }
  if (left) atomicAdd(n_unassigned, left);
}

__global__ void k_pmisr_finalize(int n, int8_t* cf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (cf[i] == 0) cf[i] = kC;
}

// ------------------------------------------------------------------------------------------
// Step 1c: DDC, Algorithm 2.  theta_i = sum_{j in F, j != i} |a_ij| / |a_ii| (ascending column
// order; +inf for a zero diagonal with a nonzero sum).  Candidates: F with theta != 0.
// k = floor(fraction |F|) capped by the candidates; tau = k-th largest candidate theta (exact
// radix select on the bit patterns of the positive doubles); candidates with theta >= tau -> C.
// ------------------------------------------------------------------------------------------
__global__ void k_ddc_theta(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                            const int8_t* __restrict__ cf, double* __restrict__ theta, int* counts) {
  int nf = 0, nc = 0;
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    double th = 0.0;
    if (cf[i] == kF) {
      double sum = 0.0, d = 0.0;
      const int e = rp[i + 1];
      // batches of kGB entries: the column loads, then the gathers, are issued together
      for (int k0 = rp[i]; k0 < e; k0 += kGB) {
        int j[kGB];
        double a[kGB];
        int8_t f[kGB];
#pragma unroll
        for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < e) ? ci[k0 + t] : -1;
#pragma unroll
        for (int t = 0; t < kGB; ++t) {
          a[t] = (j[t] >= 0) ? v[k0 + t] : 0.0;
          f[t] = (j[t] >= 0) ? cf[j[t]] : (int8_t)0;
        }
#pragma unroll
        for (int t = 0; t < kGB; ++t) {
          if (j[t] == i) d = fabs(a[t]);
          else if (j[t] >= 0 && f[t] == kF) sum += fabs(a[t]);
        }
      }      th = (sum == 0.0) ? 0.0 : sum / d;
      nf++;
      nc += (th != 0.0);
    }
    theta[i] = th;
  }
  if (nf) atomicAdd(counts, nf);
  if (nc) atomicAdd(counts + 1, nc);
}

int ddc_theta(const DCsr& A, const int8_t* cf, double* theta, Arena& tmp, cudaStream_t s) {
  const int n = A.nrows;
  int* ctr;
  AIRG_TRY(tmp.alloc(&ctr, 4));
  CU_TRY(cudaMemsetAsync(ctr, 0, sizeof(int) * 4, s));
  if (n > 0) airg::note_launch(), k_ddc_theta<<<GRID(n)>>>(n, A.rp, A.ci, A.v, cf, theta, ctr);
  KERNEL_CHECK();
  return AIRG_OK;
}

struct RadixState {
  unsigned long long prefix, mask;
  long long krem;
  long long k;  // number of candidates to convert (0: DDC converts nothing)
};

// k = floor(fraction |F|) capped by the number of candidates (ctr[0] = |F|, ctr[1] = candidates)
__global__ void k_ddc_init(const int* __restrict__ ctr, double fraction, RadixState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long k = (long long)floor(fraction * (double)ctr[0]);
    if (k > ctr[1]) k = ctr[1];
    st->prefix = 0ULL;
    st->mask = 0ULL;
    st->krem = k;
    st->k = k;
  }
}

__global__ void k_radix_hist(int n, const int8_t* __restrict__ cf, const double* __restrict__ theta,
                             const RadixState* st, int shift, unsigned* hist) {
  __shared__ unsigned sh[256];
  if (st->k <= 0) return;
  for (int t = threadIdx.x; t < 256; t += blockDim.x) sh[t] = 0;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double th = theta[i];
    if (cf[i] != kF || th == 0.0) continue;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(th);
    if ((bits & mask) == prefix) atomicAdd(&sh[(bits >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (sh[t]) atomicAdd(hist + t, sh[t]);
}

__global__ void k_radix_pick(RadixState* st, int shift, unsigned* hist) {
  if (st->k <= 0) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long cum = 0;
    int d = 0;
    for (d = 255; d >= 0; --d) {
      if (cum + (long long)hist[d] >= st->krem) break;
      cum += hist[d];
    }
    if (d < 0) d = 0;
    st->krem -= cum;
    st->prefix |= ((unsigned long long)d) << shift;
    st->mask |= 255ULL << shift;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
}

// The eight passes of the radix select in one CTA (small levels: one launch instead of sixteen);
// the digit rule is k_radix_pick's.
__global__ void __launch_bounds__(1024) k_radix_single(int n, const int8_t* __restrict__ cf,
                                                       const double* __restrict__ theta, RadixState* st) {
  __shared__ unsigned sh[256];
  __shared__ unsigned long long prefix, mask;
  __shared__ long long krem;
  if (st->k <= 0) return;
  if (threadIdx.x == 0) {
    prefix = st->prefix;
    mask = st->mask;
    krem = st->krem;
  }
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) sh[t] = 0;
    __syncthreads();
    const unsigned long long pf = prefix, mk = mask;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(theta[i]);
      if (cf[i] != kF || bits == 0ULL) continue;
      if ((bits & mk) == pf) atomicAdd(&sh[(bits >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long cum = 0;
      int d = 0;
      for (d = 255; d >= 0; --d) {
        if (cum + (long long)sh[d] >= krem) break;
        cum += sh[d];
      }
      if (d < 0) d = 0;
      krem -= cum;
      prefix |= ((unsigned long long)d) << shift;
      mask |= 255ULL << shift;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->prefix = prefix;
    st->mask = mask;
    st->krem = krem;
  }
}

__global__ void k_ddc_apply(int n, int8_t* __restrict__ cf, const double* __restrict__ theta, const RadixState* st,
                            int* converted) {
  if (st->k <= 0) return;
  const long long tau = (long long)st->prefix;  // bits of the selected (positive) theta
  int cnt = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long th = __double_as_longlong(theta[i]);  // theta >= 0
    if (cf[i] == kF && th != 0 && th >= tau) { cf[i] = kC; cnt++; }
  }
  if (cnt) atomicAdd(converted, cnt);
}

int cf_split(const DCsr& A, const SetupParams& p, int level, int8_t* cf, uint8_t* strong_out, int* nf_out,
             Arena& tmp, cudaStream_t s) {
  const int n = A.nrows;
  if (n == 0) { *nf_out = 0; return AIRG_OK; }
  uint8_t* strong = strong_out;
  if (!strong) AIRG_TRY(tmp.alloc(&strong, A.nnz));
  int *nS, *nST, *rpT, *cursor, *colT, *ctr;
  AIRG_TRY(tmp.alloc(&nS, n));
  AIRG_TRY(tmp.alloc(&nST, n));
  AIRG_TRY(tmp.alloc(&rpT, (size_t)n + 1));
  AIRG_TRY(tmp.alloc(&cursor, n));
  AIRG_TRY(tmp.alloc(&ctr, 4));
  CU_TRY(cudaMemsetAsync(nST, 0, sizeof(int) * n, s));
  CU_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * n, s));
  CU_TRY(cudaMemsetAsync(ctr, 0, sizeof(int) * 4, s));
  airg::note_launch(), k_strength<<<GRID(n)>>>(n, A.rp, A.ci, A.v, p.strong_threshold, strong, nS);
  airg::note_launch(), k_strong_T_count<<<GRID(n)>>>(n, A.rp, A.ci, strong, nST);
  KERNEL_CHECK();
  // S^T has as many entries as S, at most nnz(A): no need to read the count back
  AIRG_TRY(scan_i32(nST, rpT, n, tmp, s, nullptr));
  AIRG_TRY(tmp.alloc(&colT, (size_t)std::max(A.nnz, 1)));
  airg::note_launch(), k_strong_T_fill<<<GRID(n)>>>(n, A.rp, A.ci, strong, rpT, cursor, colT);
  double* w;
  uint8_t* D;
  AIRG_TRY(tmp.alloc(&w, n));
  AIRG_TRY(tmp.alloc(&D, n));
  airg::note_launch(), k_pmisr_init<<<GRID(n)>>>(n, nS, nST, sm64_key(p.seed, level, 0), w, cf);
  KERNEL_CHECK();
  for (int loop = 1;; ++loop) {
    if (p.pmisr_max_loops > 0 && loop > p.pmisr_max_loops) break;
    CU_TRY(cudaMemsetAsync(ctr, 0, sizeof(int), s));
    airg::note_launch(), k_pmisr_select<<<GRID(n)>>>(n, A.rp, A.ci, strong, rpT, colT, w, cf, D);
    airg::note_launch(), k_pmisr_apply<<<GRID(n)>>>(n, A.rp, A.ci, strong, rpT, colT, D, cf, ctr);
    KERNEL_CHECK();
    if (p.pmisr_max_loops <= 0) {  // uncapped: loop until nothing is left
      int left = 0;
      CU_TRY(cudaMemcpyAsync(&left, ctr, sizeof(int), cudaMemcpyDeviceToHost, s));
      CU_TRY(cudaStreamSynchronize(s));
      if (left == 0) break;
    }
  }
  airg::note_launch(), k_pmisr_finalize<<<GRID(n)>>>(n, cf);
  // DDC
  double* theta;
  AIRG_TRY(tmp.alloc(&theta, n));
  CU_TRY(cudaMemsetAsync(ctr, 0, sizeof(int) * 4, s));
  airg::note_launch(), k_ddc_theta<<<GRID(n)>>>(n, A.rp, A.ci, A.v, cf, theta, ctr);
  KERNEL_CHECK();
  // tau by radix select, all on the device (k = 0 leaves every F-point in place)
  RadixState* st;
  unsigned* hist;
  AIRG_TRY(tmp.alloc(&st, 1));
  AIRG_TRY(tmp.alloc(&hist, 256));
  CU_TRY(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned), s));
  airg::note_launch(), k_ddc_init<<<1, 32, 0, s>>>(ctr, p.ddc_fraction, st);
  if (n <= 65536) {
    airg::note_launch(), k_radix_single<<<1, 1024, 0, s>>>(n, cf, theta, st);
  } else {
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 56 - 8 * pass;
      airg::note_launch(), k_radix_hist<<<GRID(n)>>>(n, cf, theta, st, shift, hist);
      airg::note_launch(), k_radix_pick<<<1, 256, 0, s>>>(st, shift, hist);
    }
  }
  airg::note_launch(), k_ddc_apply<<<GRID(n)>>>(n, cf, theta, st, ctr + 2);
  KERNEL_CHECK();
  int hc[3];
  CU_TRY(cudaMemcpyAsync(hc, ctr, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaStreamSynchronize(s));
  const long long nF = hc[0];
  const int converted = hc[2];
  *nf_out = (int)(nF - converted);
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Step 2: stable F/C renumbering and block extraction
// ------------------------------------------------------------------------------------------
__global__ void k_isF(int n, const int8_t* __restrict__ cf, int* __restrict__ f) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    f[i] = cf[i] == kF;
}

int reuse_split(const DCsr& A, const SetupParams& p, const int8_t* cf_in, int8_t* cf, uint8_t* strong, int* nf_out,
                Arena& tmp, cudaStream_t s) {
  const int n = A.nrows;
  CU_TRY(cudaMemcpyAsync(cf, cf_in, (size_t)n, cudaMemcpyDeviceToDevice, s));
  int *nS, *isF, *fpos;
  AIRG_TRY(tmp.alloc(&nS, std::max(n, 1)));
  AIRG_TRY(tmp.alloc(&isF, std::max(n, 1)));
  AIRG_TRY(tmp.alloc(&fpos, (size_t)n + 1));
  if (n > 0) {
    airg::note_launch(), k_strength<<<GRID(n)>>>(n, A.rp, A.ci, A.v, p.strong_threshold, strong, nS);
    airg::note_launch(), k_isF<<<GRID(n)>>>(n, cf, isF);
  }
  KERNEL_CHECK();
  long long nf = 0;
  AIRG_TRY(scan_i32(isF, fpos, n, tmp, s, &nf));  // synchronises
  *nf_out = (int)nf;
  return AIRG_OK;
}
// fpos: exclusive scan of isF.  pos(i) = F ? fpos(i) : nf + (i - fpos(i)).
__global__ void k_cf_maps(int n, int nf, const int8_t* __restrict__ cf, const int* __restrict__ fpos, int* __restrict__ pos,
                          int* __restrict__ Fnat, int* __restrict__ Cnat) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    const int fp = fpos[i];
    if (cf[i] == kF) { pos[i] = fp; Fnat[fp] = i; }
    else { pos[i] = nf + (i - fp); Cnat[i - fp] = i; }
  }
}
__global__ void k_extract_count(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int8_t* __restrict__ cf,
                                const int* __restrict__ fpos, int* __restrict__ cFF, int* __restrict__ cFC,
                                int* __restrict__ cCF) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    int nFcol = 0, nCcol = 0;
    const int e = rp[i + 1];
    for (int k0 = rp[i]; k0 < e; k0 += kGB) {
      int j[kGB];
#pragma unroll
      for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < e) ? ci[k0 + t] : -1;
#pragma unroll
      for (int t = 0; t < kGB; ++t)
        if (j[t] >= 0) {
          if (cf[j[t]] == kF) nFcol++;
          else nCcol++;
        }
    }
    const int fp = fpos[i];
    if (cf[i] == kF) { cFF[fp] = nFcol; cFC[fp] = nCcol; }
    else cCF[i - fp] = nFcol;
  }
}
__global__ void k_extract_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                               const int8_t* __restrict__ cf, const int* __restrict__ fpos, DCsr Aff, DCsr Afc, DCsr Acf) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    const int fp = fpos[i];
    const bool rowF = cf[i] == kF;
    int a = rowF ? Aff.rp[fp] : Acf.rp[i - fp];
    int b = rowF ? Afc.rp[fp] : 0;
    const int e = rp[i + 1];
    for (int k0 = rp[i]; k0 < e; k0 += kGB) {
      int j[kGB], fj[kGB];
      int8_t c[kGB];
      double vv[kGB];
#pragma unroll
      for (int t = 0; t < kGB; ++t) j[t] = (k0 + t < e) ? ci[k0 + t] : -1;
#pragma unroll
      for (int t = 0; t < kGB; ++t) {
        c[t] = (j[t] >= 0) ? cf[j[t]] : (int8_t)0;
        fj[t] = (j[t] >= 0) ? fpos[j[t]] : 0;
        vv[t] = (j[t] >= 0) ? v[k0 + t] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < kGB; ++t) {
        if (j[t] < 0) continue;
        if (rowF) {
          if (c[t] == kF) { Aff.ci[a] = fj[t]; Aff.v[a++] = vv[t]; }
          else { Afc.ci[b] = j[t] - fj[t]; Afc.v[b++] = vv[t]; }
        } else if (c[t] == kF) {
          Acf.ci[a] = fj[t];
          Acf.v[a++] = vv[t];
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Steps 3-6: GMRES polynomial coefficients
// ------------------------------------------------------------------------------------------
// Box-Muller rhs in single precision (the paper asks for a normally distributed rhs of zero mean;
// FP64 log and cos would cost this kernel ~50 FP64 instructions per entry on sm_103a).  Entry i
// takes the top 24 bits k1, k2 of stream outputs 2i and 2i+1: u1 = 1 - k1 2^-24, u2 = k2 2^-24,
// z = sqrt(-2 ln u1) cos(2 pi u2), with ln and cos by fixed float sequences (written with
// explicitly rounded intrinsics, so no contraction changes them):
//  - ln x: x = m 2^e, m in [1, 2) halved above sqrt 2; f = m - 1, s = f / (2 + f);
//    ln(1 + f) = 2 atanh s = 2 (s + s^3/3 + ... + s^11/11) (Abramowitz & Stegun 4.1.28), Horner in
//    s^2; plus e ln 2 with ln 2 split into a short high part and a low part.
//  - cos 2 pi u: the nearest quarter turn q is removed in integers (|r| <= 1/8), x = 2 pi r;
//    Taylor series of cos (to x^10) and sin (to x^9) in x^2; cos(x + q pi/2) by q mod 4.
__device__ __forceinline__ uint32_t sm64_u24(uint64_t key, uint64_t c) {
  return (uint32_t)(sm64_mix(key + kGamma * (c + 1)) >> 40);
}
__device__ __forceinline__ float bm_ln(float x) {
  const uint32_t bits = __float_as_uint(x);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float f = __fsub_rn(m, 1.0f);
  const float s = __fdiv_rn(f, __fadd_rn(2.0f, f));
  const float z = __fmul_rn(s, s);
  float p = __fmaf_rn(z, 0x1.745d18p-3f, 0x1.c71c72p-3f);
  p = __fmaf_rn(z, p, 0x1.24924ap-2f);
  p = __fmaf_rn(z, p, 0x1.99999ap-2f);
  p = __fmaf_rn(z, p, 0x1.555556p-1f);
  const float r = __fmaf_rn(__fmul_rn(s, z), p, __fmul_rn(2.0f, s));
  const float ef = __int2float_rn(e);
  return __fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, r));
}
__device__ __forceinline__ float bm_cos2pi(uint32_t k) {
  const uint32_t q = (k + (1u << 21)) >> 22;
  const int ri = (int)k - (int)(q << 22);
  const float x = __fmul_rn(__fmul_rn(__int2float_rn(ri), 0x1p-24f), 0x1.921fb6p+2f);
  const float x2 = __fmul_rn(x, x);
  float c = __fmaf_rn(x2, -0x1.27e4fcp-22f, 0x1.a01a02p-16f);
  c = __fmaf_rn(x2, c, -0x1.6c16c2p-10f);
  c = __fmaf_rn(x2, c, 0x1.555556p-5f);
  c = __fmaf_rn(x2, c, -0.5f);
  c = __fmaf_rn(x2, c, 1.0f);
  float sn = __fmaf_rn(x2, 0x1.71de3ap-19f, -0x1.a01a02p-13f);
  sn = __fmaf_rn(x2, sn, 0x1.111112p-7f);
  sn = __fmaf_rn(x2, sn, -0x1.555556p-3f);
  sn = __fmaf_rn(__fmul_rn(x, x2), sn, x);
  const uint32_t qq = q & 3u;
  return qq == 0 ? c : (qq == 1 ? -sn : (qq == 2 ? -c : sn));
}
__global__ void k_box_muller(int n, uint64_t key, double* __restrict__ z) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t k1 = sm64_u24(key, 2 * (uint64_t)i), k2 = sm64_u24(key, 2 * (uint64_t)i + 1);
    const float u1 = __fsub_rn(1.0f, __fmul_rn(__uint2float_rn(k1), 0x1p-24f));
    const float t = __fmul_rn(-2.0f, bm_ln(u1));
    z[i] = (double)__fmul_rn(__fsqrt_rn(t), bm_cos2pi(k2));
  }
}

// TSQR of the tall power basis and the least-squares fit (setup steps 4-6), in one launch.
//
// One warp factors a tile of 32*RPL rows x C columns held entirely in registers (lane l owns rows
// l, l+32, ...) by C Householder reflections, leaving the C x C upper-triangular factor in row k of
// lane k.  Stage 0 tiles the basis; each later stage stacks G = 32*RPLC/C factors of the previous
// stage and factors them again.  The warp that completes a group (the last of its G producers to
// arrive, counted with an atomic after a fence) combines it, so the whole tree runs in the one
// launch with no waiting; the warp that produces the single final factor also solves the small
// least-squares problem.  The combination order is fixed by the tile numbering, so the result does
// not depend on which warp arrives last.  Rows past n and columns past ncols are zero (appended
// zero columns leave the leading ncols x ncols block of R unchanged, so bases of up to 4, 8 or 16
// columns share the C = 4, 8, 16 instances).
//
// FP64 issue, not bandwidth, bounds this kernel on sm_103a (one warp-wide FP64 instruction per
// about 64 clocks per SM sub-partition), so each reflection takes one warp reduction of all C dots
// by recursive halving (about C+1 additions per lane instead of 5 per dot): the dots x.M_j of the
// column x = M(k:, k) with the columns j >= k (j = k gives ||x||^2); with v = x - a e_k,
// v.M_j = x.M_j - a M(k, j) and ||v||^2 = 2 |a| (|a| + |x_k|).
constexpr int kQrMaxCols = 16;

// Sum over the 32 lanes of p[0..N) (N = 4, 8 or 16), returned to every lane in p.
template <int N>
__device__ __forceinline__ void warp_sum_vec(double (&p)[N], int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  // recursive halving: after the levels xor 16, 8, ... each lane holds one partial sum
  double q[N];
#pragma unroll
  for (int j = 0; j < N; ++j) q[j] = p[j];
  int width = N;
#pragma unroll
  for (int bit = 4; bit >= 0 && width > 1; --bit) {
    const bool upper = (lane >> bit) & 1;
    const int h = width >> 1;
#pragma unroll
    for (int j = 0; j < N / 2; ++j) {
      if (j < h) {
        const double keep = upper ? q[j + h] : q[j];
        const double send = upper ? q[j] : q[j + h];
        q[j] = keep + __shfl_xor_sync(FULL, send, 1 << bit);
      }
    }
    width = h;
  }
  // remaining levels on the single value
  constexpr int LG = (N == 4) ? 2 : (N == 8 ? 3 : 4);
#pragma unroll
  for (int bit = 4 - LG; bit >= 0; --bit) q[0] += __shfl_xor_sync(FULL, q[0], 1 << bit);
  // lane l now holds the total of index (l >> (5 - LG)); gather all of them
#pragma unroll
  for (int j = 0; j < N; ++j) p[j] = __shfl_sync(FULL, q[0], j << (5 - LG));
}

template <int C, int RPL>
__device__ __forceinline__ void house_warp(double (&M)[RPL][C], int lane) {
  constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < C; ++k) {
    double p[C];
#pragma unroll
    for (int j = 0; j < C; ++j) p[j] = 0.0;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      if (q > 0 || lane >= k) {
        const double x = M[q][k];
#pragma unroll
        for (int j = k; j < C; ++j) p[j] = fma(x, M[q][j], p[j]);
      }
    }
    warp_sum_vec<C>(p, lane);
    const double x0 = __shfl_sync(FULL, M[0][k], k);
    const double xn = sqrt(p[k]);
    const double a = (x0 >= 0.0) ? -xn : xn;
    const double vn2 = 2.0 * xn * (xn + fabs(x0));
    if (vn2 > 0.0) {
      const double two_over = 2.0 / vn2;
      // v = x - a e_k: lane k's first-row entry of v is x0 - a, the rest are x's own entries; one
      // FMA per row with the operand selected (an FP64 instruction costs its full pipe time on
      // sm_103a however many lanes it has)
      const double v0 = (lane == k) ? x0 - a : M[0][k];
#pragma unroll
      for (int j = k + 1; j < C; ++j) {
        const double mkj = __shfl_sync(FULL, M[0][j], k);
        const double f = (p[j] - a * mkj) * two_over;
        if (lane >= k) M[0][j] = fma(-f, v0, M[0][j]);
#pragma unroll
        for (int q = 1; q < RPL; ++q) M[q][j] = fma(-f, M[q][k], M[q][j]);
      }
    }
    if (lane == k) M[0][k] = a;
  }
}

// Least squares min || beta e1 - R(:, 2:end) y || (setup step 6), breakdown truncation when
// |R_cc| <= 1e-12 ||R(:,c)||, Givens rotations and back substitution.  One thread.  R is row-major
// with leading dimension ld >= m + 1.
__device__ void poly_lsq(const double* R, int ld, int m, double* __restrict__ alpha, int* fitted) {
  const int nc = ld;
  int mf = m;
  for (int c = 1; c <= m; ++c) {
    double cn = 0.0;
    for (int r = 0; r <= c; ++r) cn += R[r * nc + c] * R[r * nc + c];
    cn = sqrt(cn);
    if (!(fabs(R[c * nc + c]) > 1e-12 * cn)) { mf = c; break; }
  }
  double H[kQrMaxCols + 1][kQrMaxCols];
  double g[kQrMaxCols + 1];
  for (int i = 0; i <= mf; ++i) {
    g[i] = 0.0;
    for (int j = 0; j < mf; ++j) H[i][j] = R[i * nc + j + 1];
  }
  g[0] = R[0];
  for (int k = 0; k < mf; ++k) {
    const double a = H[k][k], b = H[k + 1][k];
    const double d = hypot(a, b);
    double c_ = 1.0, s_ = 0.0;
    if (d != 0.0) { c_ = a / d; s_ = b / d; }
    for (int j = k; j < mf; ++j) {
      const double t1 = H[k][j], t2 = H[k + 1][j];
      H[k][j] = c_ * t1 + s_ * t2;
      H[k + 1][j] = -s_ * t1 + c_ * t2;
    }
    const double t1 = g[k], t2 = g[k + 1];
    g[k] = c_ * t1 + s_ * t2;
    g[k + 1] = -s_ * t1 + c_ * t2;
  }
  for (int i = 0; i < m; ++i) alpha[i] = 0.0;
  for (int i = mf - 1; i >= 0; --i) {
    double sum = g[i];
    for (int j = i + 1; j < mf; ++j) sum -= H[i][j] * alpha[j];
    alpha[i] = (H[i][i] != 0.0) ? sum / H[i][i] : 0.0;
  }
  *fitted = mf;
}

constexpr int kTsqrMaxStages = 16;
struct TsqrPlan {
  int nstages;                       // stage 0 tiles the basis
  long long ntiles[kTsqrMaxStages];  // tiles (= factors produced) per stage
  long long foff[kTsqrMaxStages];    // offset of the stage's factors in the factor buffer (doubles)
  long long coff[kTsqrMaxStages];    // offset of the stage's group counters (stages >= 1)
};

template <int C, int RPL>
__device__ __forceinline__ void store_factor(const double (&M)[RPL][C], int lane, double* o) {
  if (lane < C) {
#pragma unroll
    for (int j = 0; j < C; ++j) o[lane * C + j] = (j >= lane) ? M[0][j] : 0.0;
  }
}

template <int C, int RPL, int RPLC>
__global__ void __launch_bounds__(256) k_tsqr(const double* __restrict__ K, long long n, int ncols, TsqrPlan plan,
                                              double* fbuf, unsigned* cnt, int m, double* __restrict__ alpha,
                                              int* __restrict__ fitted) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int G = 32 * RPLC / C;  // factors per combined tile
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= plan.ntiles[0]) return;  // the whole warp leaves together
  {
    double M[RPL][C];
    const long long r0 = w * (32LL * RPL);
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const long long r = r0 + lane + 32 * q;
#pragma unroll
      for (int c = 0; c < C; ++c) M[q][c] = (r < n && c < ncols) ? K[(long long)c * n + r] : 0.0;
    }
    house_warp<C, RPL>(M, lane);
    store_factor<C, RPL>(M, lane, fbuf + plan.foff[0] + w * C * C);
  }
  long long t = w;
  for (int s = 1; s < plan.nstages; ++s) {
    __threadfence();
    __syncwarp();
    const long long g = t / G, first = g * G;
    const long long left = plan.ntiles[s - 1] - first;
    const int gs = (int)(left < G ? left : G);
    unsigned prev = 0;
    if (lane == 0) prev = atomicAdd(cnt + plan.coff[s] + g, 1u);
    prev = __shfl_sync(FULL, prev, 0);
    if (prev != (unsigned)(gs - 1)) return;  // another producer of this group combines it
    __threadfence();
    double M[RPLC][C];
    const double* src = fbuf + plan.foff[s - 1] + first * C * C;  // gs stacked C x C factors, row-major
#pragma unroll
    for (int q = 0; q < RPLC; ++q) {
      const int r = lane + 32 * q;
#pragma unroll
      for (int c = 0; c < C; ++c) M[q][c] = (r < gs * C) ? __ldcg(src + (long long)r * C + c) : 0.0;
    }
    house_warp<C, RPLC>(M, lane);
    store_factor<C, RPLC>(M, lane, fbuf + plan.foff[s] + g * C * C);
    t = g;
  }
  __syncwarp();
  if (lane == 0) poly_lsq(fbuf + plan.foff[plan.nstages - 1], C, m, alpha, fitted);
}

// Column count of the register QR instance for an nc-column basis.
int tsqr_cols(int nc) { return nc <= 4 ? 4 : (nc <= 8 ? 8 : 16); }

template <int C, int RPL, int RPLC>
int tsqr_run(const double* K, long long n, int nc, int m, double* alpha, int* fitted, Arena& tmp, cudaStream_t s) {
  constexpr int G = 32 * RPLC / C;
  TsqrPlan plan{};
  long long nt = (n + 32LL * RPL - 1) / (32LL * RPL);
  long long ftot = 0, ctot = 0;
  int ns = 0;
  for (;;) {
    if (ns >= kTsqrMaxStages) return AIRG_ERR_UNSUPPORTED;
    plan.ntiles[ns] = nt;
    plan.foff[ns] = ftot;
    ftot += nt * C * C;
    plan.coff[ns] = ctot;
    if (ns > 0) ctot += nt;
    ++ns;
    if (nt == 1) break;
    nt = (nt + G - 1) / G;
  }
  plan.nstages = ns;
  double* fbuf;
  unsigned* cnt;
  AIRG_TRY(tmp.alloc(&fbuf, (size_t)ftot));
  AIRG_TRY(tmp.alloc(&cnt, (size_t)std::max(1LL, ctot)));
  if (ctot > 0) CU_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (size_t)ctot, s));
  // The tiles are independent warps.  In an 8-warp CTA the eight tiles of a combine group finish
  // together and the last of them then combines the group alone, holding the CTA's slot with one
  // warp busy; with single-warp CTAs the seven finished warps' slots take new tiles at once.  The
  // resident warps are the same (registers come from each sub-partition's quarter of the file:
  // two warps of 170 registers a sub-partition either way), but the FP64 pipe is busy 83 % instead
  // of 68 % of the active cycles on the 8-row instance (20 % faster on the largest levels).  The
  // 2-row instances lost time to the extra CTA launches, so they keep 8 warps a CTA.
  constexpr int warps = RPL >= 4 ? 1 : 8;
  const long long blocks = (plan.ntiles[0] + warps - 1) / warps;
  if (blocks > 0x7fffffffLL) return AIRG_ERR_UNSUPPORTED;
  airg::note_launch(), k_tsqr<C, RPL, RPLC><<<(unsigned)blocks, 32 * warps, 0, s>>>(K, n, nc, plan, fbuf, cnt, m, alpha, fitted);
  return cuda_status(cudaGetLastError());
}

// Leaf tiles of 32*RPL rows: 8 rows per lane once the basis has enough rows to give every SM
// sub-partition a few warps, else 2 (shorter FP64 chains per warp on small levels).
int tsqr_fit(const double* K, long long n, int nc, int m, double* alpha, int* fitted, Arena& tmp, cudaStream_t s) {
  const bool big = n >= 152LL * 8 * 256;
  switch (tsqr_cols(nc)) {
    case 4: return big ? tsqr_run<4, 8, 2>(K, n, nc, m, alpha, fitted, tmp, s) : tsqr_run<4, 2, 2>(K, n, nc, m, alpha, fitted, tmp, s);
    case 8: return big ? tsqr_run<8, 8, 2>(K, n, nc, m, alpha, fitted, tmp, s) : tsqr_run<8, 2, 2>(K, n, nc, m, alpha, fitted, tmp, s);
    default: return big ? tsqr_run<16, 4, 2>(K, n, nc, m, alpha, fitted, tmp, s) : tsqr_run<16, 2, 2>(K, n, nc, m, alpha, fitted, tmp, s);
  }
}

int poly_fit(const DCsr& A, int m, uint64_t seed, int level, double* alpha, int* fitted, Arena& tmp,
             cudaStream_t s) {
  const int n = A.nrows, nc = m + 1;
  if (m < 1 || nc > kQrMaxCols) return AIRG_ERR_ARG;
  if (n == 0) {
    CU_TRY(cudaMemsetAsync(alpha, 0, sizeof(double) * m, s));
    CU_TRY(cudaMemsetAsync(fitted, 0, sizeof(int), s));
    return AIRG_OK;
  }
  double* K;
  AIRG_TRY(tmp.alloc(&K, (size_t)n * nc));
  airg::note_launch(), k_box_muller<<<GRID(n)>>>(n, sm64_key(seed, level, 1), K);
  KERNEL_CHECK();
  const int lanes = pick_lanes((double)A.nnz / std::max(1, n));
  for (int c = 1; c < nc; ++c) AIRG_TRY(dev_spmv(A, K + (size_t)(c - 1) * n, nullptr, K + (size_t)c * n, SPMV_SET, lanes, s));
  // the fitted count stays on the device (read back once the hierarchy is built): no host
  // synchronisation here, so the work queued after the fit (the side stream's P and A P) overlaps it
  AIRG_TRY(tsqr_fit(K, n, nc, m, alpha, fitted, tmp, s));
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Steps 7-8: first-order fixed-sparsity powers (eq. fixed_sparsity), one thread per entry.
//   P1 = A;  P_p(i,j) = sum_{l in S_i ascending} P_{p-1}(i,l) a_lj   (fma; l with no a_lj skipped)
//   Ainv(i,j) = alpha_0 delta_ij + alpha_1 P1(i,j) + ... accumulated left to right with fma.
// ------------------------------------------------------------------------------------------
__global__ void k_row_index(int n, const int* __restrict__ rp, int* __restrict__ rowidx) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k) rowidx[k] = (int)i;
}

__device__ __forceinline__ int find_col(const int* __restrict__ ci, int b, int e, int j) {
  while (b < e) {
    const int mid = (b + e) >> 1;
    const int c = ci[mid];
    if (c < j) b = mid + 1;
    else if (c > j) e = mid;
    else return mid;
  }
  return -1;
}

__global__ void k_fs_init(int nnz, const int* __restrict__ rowidx, const int* __restrict__ ci,
                          const double* __restrict__ v, const double* __restrict__ alpha, int m,
                          double* __restrict__ ainv) {
  const double a0 = alpha[0];
  const double a1 = m > 1 ? alpha[1] : 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    double acc = (ci[k] == rowidx[k]) ? a0 : 0.0;
    if (m > 1) acc = fma(a1, v[k], acc);
    ainv[k] = acc;
  }
}

// For entry k = (i, j) of the pattern and each q in row i (l = ci[q]), the position of a_lj in row
// l, or -1: the gather the paper describes as done once, after which every power reads it.
// Row i's block of the index holds r_i x r_i entries (r_i = row length) at base[i].
__global__ void k_fs_rowsq(int n, const int* __restrict__ rp, long long* __restrict__ sq) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long r = rp[i + 1] - rp[i];
    sq[i] = r * r;
  }
}
__global__ void k_fs_gather(int nnz, const int* __restrict__ rowidx, const int* __restrict__ prp,
                            const int* __restrict__ pci, const int* __restrict__ arp, const int* __restrict__ aci,
                            const long long* __restrict__ ntot, long long cap, const long long* __restrict__ base,
                            int* __restrict__ idx) {
  if (*ntot > cap) return;  // too large: the powers search instead
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const int i = rowidx[k], j = pci[k];
    const int b = prp[i], r = prp[i + 1] - b;
    int* o = idx + base[i] + (long long)(k - b) * r;
    for (int q = 0; q < r; ++q) {
      const int l = pci[b + q];
      o[q] = find_col(aci, arp[l], arp[l + 1], j);
    }
  }
}
// Values of A on a larger pattern P (second-order sparsity): a_ij where A has the entry, else 0.
__global__ void k_fs_scatter(int nnz, const int* __restrict__ rowidx, const int* __restrict__ pci,
                             const int* __restrict__ arp, const int* __restrict__ aci, const double* __restrict__ av,
                             double* __restrict__ p1) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const int i = rowidx[k];
    const int t = find_col(aci, arp[i], arp[i + 1], pci[k]);
    p1[k] = t >= 0 ? av[t] : 0.0;
  }
}
__global__ void k_fs_power(int nnz, const int* __restrict__ rowidx, const int* __restrict__ prp,
                           const int* __restrict__ pci, const int* __restrict__ arp, const int* __restrict__ aci,
                           const long long* __restrict__ ntot, long long cap, const long long* __restrict__ base,
                           const int* __restrict__ idx, const double* __restrict__ av, const double* __restrict__ prev,
                           double* __restrict__ cur, double* __restrict__ ainv, const double* __restrict__ alpha_p) {
  const double ap = *alpha_p;
  const bool gathered = *ntot <= cap;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x) {
    const int i = rowidx[k];
    const int b = prp[i], r = prp[i + 1] - b;
    double acc = 0.0;
    if (gathered) {
      const int* g = idx + base[i] + (long long)(k - b) * r;
      for (int q = 0; q < r; ++q) {
        const int t = g[q];
        if (t >= 0) acc = fma(prev[b + q], av[t], acc);
      }
    } else {  // rows of hundreds of entries (dense coarse levels): search every position
      const int j = pci[k];
      for (int q = b; q < b + r; ++q) {
        const int l = pci[q];
        const int t = find_col(aci, arp[l], arp[l + 1], j);
        if (t >= 0) acc = fma(prev[q], av[t], acc);
      }
    }
    cur[k] = acc;
    ainv[k] = fma(ap, acc, ainv[k]);
  }
}

int fixed_sparsity_inverse(const DCsr& A, const double* alpha, int m, DCsr& out, Arena& own, Arena& tmp,
                           cudaStream_t s, int order) {
  const int n = A.nrows;
  // the pattern P of the powers: A's own (first order) or that of A^2 (second order); A has its
  // diagonal, so pattern(A^2) contains pattern(A)
  DCsr Pt = A;
  if (order >= 2 && A.nnz > 0) AIRG_TRY(spgemm(A, A, 1.0, 0.0, false, Pt, tmp, tmp, s));
  const int nnz = Pt.nnz;
  AIRG_TRY(own.csr(out, n, n, nnz));
  CU_TRY(cudaMemcpyAsync(out.rp, Pt.rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
  CU_TRY(cudaMemcpyAsync(out.ci, Pt.ci, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, s));
  if (nnz == 0) return AIRG_OK;
  int* rowidx;
  AIRG_TRY(tmp.alloc(&rowidx, nnz));
  airg::note_launch(), k_row_index<<<GRID(n)>>>(n, Pt.rp, rowidx);
  const double* p1 = A.v;  // tilde(A^1): A on the pattern
  if (Pt.rp != A.rp) {
    double* sc;
    AIRG_TRY(tmp.alloc(&sc, nnz));
    airg::note_launch(), k_fs_scatter<<<GRID(nnz)>>>(nnz, rowidx, Pt.ci, A.rp, A.ci, A.v, sc);
    p1 = sc;
  }
  airg::note_launch(), k_fs_init<<<GRID(nnz)>>>(nnz, rowidx, Pt.ci, p1, alpha, m, out.v);
  KERNEL_CHECK();
  if (m > 2) {
    double *pa, *pb;
    long long *sq, *base;
    int* idx;
    AIRG_TRY(tmp.alloc(&pa, nnz));
    AIRG_TRY(tmp.alloc(&pb, nnz));
    AIRG_TRY(tmp.alloc(&sq, n));
    AIRG_TRY(tmp.alloc(&base, (size_t)n + 1));
    airg::note_launch(), k_fs_rowsq<<<GRID(n)>>>(n, Pt.rp, sq);
    // the gathered index costs sum_i r_i^2 ints: it is used when that is at most 128 per nonzero
    // (and 2 GiB), decided on the device from base[n]; otherwise every power searches
    AIRG_TRY(scan_i64(sq, base, n, tmp, s, nullptr));
    const long long cap = std::min(128LL * nnz, 1LL << 29);
    AIRG_TRY(tmp.alloc(&idx, (size_t)cap));
    airg::note_launch(), k_fs_gather<<<GRID(nnz)>>>(nnz, rowidx, Pt.rp, Pt.ci, A.rp, A.ci, base + n, cap, base, idx);
    KERNEL_CHECK();
    const double* prev = p1;
    double* cur = pa;
    for (int p = 2; p < m; ++p) {
      airg::note_launch(), k_fs_power<<<GRID(nnz)>>>(nnz, rowidx, Pt.rp, Pt.ci, A.rp, A.ci, base + n, cap, base, idx,
                                                     A.v, prev, cur, out.v, alpha + p);
      KERNEL_CHECK();
      prev = cur;
      cur = (cur == pa) ? pb : pa;
    }
  }
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Deterministic row-wise SpGEMM with the relative row-wise inf-norm drop (steps 9 and 11).
// Row i: candidate columns = union of B's rows named by A's row i (bitonic sort + unique in
// shared memory); each output c_ij = sum over A's row in ascending order of fma(a_il, b_lj, .)
// (b_lj by binary search); scale; drop |c| < tol * max_j |c_ij| unless (keep_diag and j == i).
// Rows whose candidate count fits kWarpCap are done by one warp, longer rows by one CTA.
// ------------------------------------------------------------------------------------------
constexpr int kWarpCap = 1024;
constexpr int kBlockCapMax = 32768;

__global__ void k_spgemm_ub(int ar, const int* __restrict__ arp, const int* __restrict__ aci,
                            const int* __restrict__ brp, const int* __restrict__ blen, long long* __restrict__ ub) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ar; i += (long long)gridDim.x * blockDim.x) {
    long long t = 0;
    for (int k = arp[i]; k < arp[i + 1]; ++k) {
      const int l = aci[k];
      t += blen ? blen[l] : brp[l + 1] - brp[l];
    }
    ub[i] = t;
  }
}

struct SpgArgs {
  int ar;
  const int *arp, *aci;
  const double* av;
  const int *brp, *bci;
  const double* bv;
  const int *bbeg, *blen;  // B in padded form (row l at bbeg[l], blen[l] entries); nullptr: CSR brp
  double scale, tol;
  int scale_mode;  // 0: scale == 1, 1: scale == -1 (a sign flip), 2: general
  int keep_diag;
  const long long* ubo;
  int* tcol;
  double* tval;
  int* cnt;
};

// Group-generic pieces (G threads cooperate; sync() is __syncwarp or __syncthreads).
template <int G>
struct Grp {
  __device__ static void sync() {
    if (G == 32) __syncwarp();
    else __syncthreads();
  }
};

template <int G>
__device__ void bitonic_sort(int* a, int P, int t) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int idx = t; idx < P; idx += G) {
        const int ixj = idx ^ j;
        if (ixj > idx) {
          const int x = a[idx], y = a[ixj];
          const bool up = ((idx & k) == 0);
          if ((x > y) == up) { a[idx] = y; a[ixj] = x; }
        }
      }
      Grp<G>::sync();
    }
}

// Removes duplicates from the sorted a[0..P) (padding 0x7fffffff at the end) in place, keeping
// order; returns the number of distinct values.  Chunks of 32 are read completely before any
// write, and the last original value of the previous chunk is carried in a register.
__device__ int warp_unique_sorted(int* a, int P, int lane) {
  int outc = 0, prev_last = -1;
  for (int base = 0; base < P; base += 32) {
    const int idx = base + lane;
    const int val = idx < P ? a[idx] : 0x7fffffff;
    int prv = __shfl_up_sync(0xffffffffu, val, 1);
    if (lane == 0) prv = prev_last;
    const bool kf = val != 0x7fffffff && val != prv;
    const unsigned bal = __ballot_sync(0xffffffffu, kf);
    prev_last = __shfl_sync(0xffffffffu, val, 31);
    __syncwarp();
    if (kf) a[outc + __popc(bal & ((1u << lane) - 1u))] = val;
    outc += __popc(bal);
    __syncwarp();
  }
  return outc;
}

// scale * x; the factors 1 and -1 are applied exactly on the integer pipe
__device__ __forceinline__ double spg_scale(const SpgArgs& g, double x) {
  if (g.scale_mode == 0) return x;
  if (g.scale_mode == 1) return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
  return g.scale * x;
}
// bit pattern of tol * max|c| from the bit pattern of max|c|; |c| < tol * max  <=>  abs_bits(c) < result
__device__ __forceinline__ long long spg_thr(const SpgArgs& g, long long mx_bits) {
  return abs_bits(g.tol * __longlong_as_double(mx_bits));
}

__device__ __forceinline__ void spg_brow(const SpgArgs& g, int l, int& b, int& e) {
  if (g.blen) {
    b = g.bbeg[l];
    e = b + g.blen[l];
  } else {
    b = g.brp[l];
    e = g.brp[l + 1];
  }
}

__device__ __forceinline__ double spg_value(const SpgArgs& g, int ab, int ae, int j) {
  double acc = 0.0;
  for (int k = ab; k < ae; ++k) {
    const int l = g.aci[k];
    int b0, b1;
    spg_brow(g, l, b0, b1);
    const int t = find_col(g.bci, b0, b1, j);
    if (t >= 0) acc = fma(g.av[k], g.bv[t], acc);
  }
  return spg_scale(g, acc);
}

// Short rows (candidate count <= kThreadCap): one thread per row.  For each A entry in ascending
// order the B row is merged into a per-thread sorted list whose accumulators take
// fma(a_il, b_lj, acc) as the entry is met, so every output sums in ascending inner index with no
// search.  Rows with more candidates go to `mid_rows` (warp kernel).
constexpr int kThreadCap = 32;

__global__ void __launch_bounds__(128) k_spgemm_thread(SpgArgs g, int* mid_rows, int* n_mid) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < g.ar; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    const long long ub = g.ubo[i + 1] - g.ubo[i];
    if (ub == 0) { g.cnt[i] = 0; continue; }
    if (ub > kThreadCap) { mid_rows[atomicAdd(n_mid, 1)] = i; continue; }
    const int ab = g.arp[i], ae = g.arp[i + 1];
    int cand[kThreadCap];
    double acc[kThreadCap];
    int u = 0;
    // A entries in batches of kGB: their columns, then their B row ranges, are loaded together
    for (int k0 = ab; k0 < ae; k0 += kGB) {
      int lb[kGB];
      double la[kGB];
      int qbs[kGB], qes[kGB];
#pragma unroll
      for (int t = 0; t < kGB; ++t) {
        lb[t] = (k0 + t < ae) ? g.aci[k0 + t] : -1;
        la[t] = (k0 + t < ae) ? g.av[k0 + t] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < kGB; ++t) {
        qbs[t] = 0;
        qes[t] = 0;
        if (lb[t] >= 0) spg_brow(g, lb[t], qbs[t], qes[t]);
      }
#pragma unroll
      for (int e = 0; e < kGB; ++e) {
      const double a = la[e];
      const int qb = qbs[e], qe = qes[e];
      for (int q = qb; q < qe; ++q) {
        const int j = g.bci[q];
        const double bv = g.bv[q];
        int pos = u;
        while (pos > 0 && cand[pos - 1] > j) --pos;
        // integer work (search, insertion) may diverge; the one FMA per product sits after it, where
        // the lanes meet again: an FP64 instruction costs sm_103a's FP64 pipe the same time with
        // few lanes as with all, so one shared FMA instead of one per branch
        if (pos > 0 && cand[pos - 1] == j) {
          --pos;
        } else {
          for (int t = u; t > pos; --t) { cand[t] = cand[t - 1]; acc[t] = acc[t - 1]; }
          cand[pos] = j;
          acc[pos] = 0.0;
          ++u;
        }
        acc[pos] = fma(a, bv, acc[pos]);
      }
      }
    }
    long long mx = 0;
    for (int t = 0; t < u; ++t) {
      acc[t] = spg_scale(g, acc[t]);
      mx = max(mx, abs_bits(acc[t]));
    }
    const long long thr = spg_thr(g, mx);
    const long long o = g.ubo[i];
    int outc = 0;
    for (int t = 0; t < u; ++t) {
      const double c = acc[t];
      const int j = cand[t];
      if (abs_bits(c) >= thr || (g.keep_diag && j == i)) {
        g.tcol[o + outc] = j;
        g.tval[o + outc] = c;
        ++outc;
      }
    }
    g.cnt[i] = outc;
  }
}

// Medium rows (candidate count <= kWarpCap): one warp per row with a shared-memory hash table.
// For each A entry (ascending, one at a time) the lanes take the distinct columns of that B row in
// parallel and update their slots with fma -- no two lanes touch one key in the same step, so every
// output accumulates in ascending inner index.  The occupied slots are then compacted, sorted by
// column (bitonic, values carried along), scaled and dropped.

template <int G>
__device__ void bitonic_sort_kv(int* a, double* v, int P, int t) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int idx = t; idx < P; idx += G) {
        const int ixj = idx ^ j;
        if (ixj > idx) {
          const int x = a[idx], y = a[ixj];
          const bool up = ((idx & k) == 0);
          if ((x > y) == up) {
            a[idx] = y;
            a[ixj] = x;
            const double tv = v[idx];
            v[idx] = v[ixj];
            v[ixj] = tv;
          }
        }
      }
      Grp<G>::sync();
    }
}

// Writes the kept entries of a warp's compacted row (key/val[0..u), u <= 32*NE) in column order:
// a kept entry's position is the number of kept columns below it (dropped entries take the key
// 0x7fffffff, which is below no kept column).  Returns the number kept.
template <int NE>
__device__ __forceinline__ int spg_rank_write(const SpgArgs& g, int* key, const double* val, int u, long long thr,
                                              int i, long long o, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  int mk[NE];
  double mv[NE];
  int kept = 0;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int t = lane + 32 * e;
    int j = 0x7fffffff;
    double c = 0.0;
    if (t < u) {
      j = key[t];
      c = val[t];
      if (!(abs_bits(c) >= thr || (g.keep_diag && j == i))) j = 0x7fffffff;
    }
    mk[e] = j;
    mv[e] = c;
    kept += __popc(__ballot_sync(FULL, j != 0x7fffffff));
  }
  __syncwarp();
#pragma unroll
  for (int e = 0; e < NE; ++e)
    if (lane + 32 * e < u) key[lane + 32 * e] = mk[e];
  __syncwarp();
  int rk[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) rk[e] = 0;
  for (int t = 0; t < u; ++t) {
    const int kt = key[t];
#pragma unroll
    for (int e = 0; e < NE; ++e) rk[e] += (kt < mk[e]);
  }
#pragma unroll
  for (int e = 0; e < NE; ++e)
    if (mk[e] != 0x7fffffff) {
      g.tcol[o + rk[e]] = mk[e];
      g.tval[o + rk[e]] = mv[e];
    }
  return kept;
}

template <int CAP, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, CAP <= 512 ? 4 : 1) k_spgemm_warp(SpgArgs g, const int* __restrict__ rows,
                                                            const int* __restrict__ nrows_dev, int* next_rows,
                                                            int* n_next, int lim) {
  __shared__ int hkey[WARPS][CAP];
  __shared__ double hval[WARPS][CAP];
  __shared__ double s_a[WARPS][32];
  __shared__ int s_b0[WARPS][32], s_len[WARPS][32];
  const int nrows = *nrows_dev;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* key = hkey[wid];
  double* val = hval[wid];
  const long long gw = (long long)blockIdx.x * WARPS + wid;
  const long long nw = (long long)gridDim.x * WARPS;
  for (long long ii = gw; ii < nrows; ii += nw) {
    const int i = rows[ii];
    const long long ub = g.ubo[i + 1] - g.ubo[i];
    if (ub > lim) {
      if (lane == 0) next_rows[atomicAdd(n_next, 1)] = i;
      continue;
    }
    int H = 32, lg = 5;
    while (H < ub) { H <<= 1; ++lg; }
    for (int t = lane; t < H; t += 32) { key[t] = -1; val[t] = 0.0; }
    __syncwarp();
    // A entries 32 at a time: their values and B row ranges are loaded by the lanes together and
    // kept in shared memory, and the first 32 candidates of the next entry are loaded while the
    // current entry's slots are updated, so the entries do not each wait on a chain of dependent
    // global loads.  The updates themselves stay one entry after another, in ascending order.
    const int ab = g.arp[i], na = g.arp[i + 1] - ab;
    double* sa = s_a[wid];
    int* sb0 = s_b0[wid];
    int* slen = s_len[wid];
    for (int e0 = 0; e0 < na; e0 += 32) {
      const int ne = min(32, na - e0);
      if (lane < ne) {
        const int l = g.aci[ab + e0 + lane];
        sa[lane] = g.av[ab + e0 + lane];
        int b0, b1;
        spg_brow(g, l, b0, b1);
        sb0[lane] = b0;
        slen[lane] = b1 - b0;
      }
      __syncwarp();
      int jn = -1;
      double bn = 0.0;
      if (lane < slen[0]) {
        jn = g.bci[sb0[0] + lane];
        bn = g.bv[sb0[0] + lane];
      }
      for (int e = 0; e < ne; ++e) {
        const double a = sa[e];
        const int b0 = sb0[e], len = slen[e];
        const int j0 = jn;
        const double bv0 = bn;
        if (e + 1 < ne) {  // next entry's first candidates
          jn = -1;
          if (lane < slen[e + 1]) {
            jn = g.bci[sb0[e + 1] + lane];
            bn = g.bv[sb0[e + 1] + lane];
          }
        }
        for (int t = lane; t < len; t += 32) {
          const int j = t < 32 ? j0 : g.bci[b0 + t];
          const double bv = t < 32 ? bv0 : g.bv[b0 + t];
          unsigned h = ((unsigned)j * 0x9E3779B1u) >> (32 - lg);
          while (true) {
            const int prev = atomicCAS(&key[h], -1, j);
            if (prev == -1 || prev == j) break;
            h = (h + 1) & (H - 1);
          }
          val[h] = fma(a, bv, val[h]);
        }
        __syncwarp();
      }
    }
    // compact occupied slots to the front (chunks read before written), then sort by column
    int u = 0;
    for (int base = 0; base < H; base += 32) {
      const int idx = base + lane;
      const int kk = key[idx];
      const double vv = val[idx];
      const bool occ = kk >= 0;
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      __syncwarp();
      if (occ) {
        const int d = u + __popc(bal & ((1u << lane) - 1u));
        key[d] = kk;
        val[d] = vv;
      }
      u += __popc(bal);
      __syncwarp();
    }
    long long mx = 0;
    for (int t = lane; t < u; t += 32) {
      const double c = spg_scale(g, val[t]);
      val[t] = c;
      mx = max(mx, abs_bits(c));
    }
    for (int s2 = 16; s2 > 0; s2 >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, s2));
    const long long thr = spg_thr(g, mx);
    const long long o = g.ubo[i];
    // drop first (the threshold is known), so that only the kept entries are ordered
    int u2 = 0;
    for (int base = 0; base < u; base += 32) {
      const int t = base + lane;
      int j = 0;
      double c = 0.0;
      bool keep = false;
      if (t < u) {
        j = key[t];
        c = val[t];
        keep = abs_bits(c) >= thr || (g.keep_diag && j == i);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) {
        const int d = u2 + __popc(bal & ((1u << lane) - 1u));
        key[d] = j;
        val[d] = c;
      }
      u2 += __popc(bal);
      __syncwarp();
    }
    if (u2 <= 256) {  // position = rank among the kept columns (every entry kept: threshold 0)
      if (u2 <= 32) spg_rank_write<1>(g, key, val, u2, 0, i, o, lane);
      else if (u2 <= 64) spg_rank_write<2>(g, key, val, u2, 0, i, o, lane);
      else if (u2 <= 128) spg_rank_write<4>(g, key, val, u2, 0, i, o, lane);
      else spg_rank_write<8>(g, key, val, u2, 0, i, o, lane);
    } else {
      int P = 32;
      while (P < u2) P <<= 1;
      for (int t = u2 + lane; t < P; t += 32) { key[t] = 0x7fffffff; val[t] = 0.0; }
      __syncwarp();
      bitonic_sort_kv<32>(key, val, P, lane);
      for (int t = lane; t < u2; t += 32) {
        g.tcol[o + t] = key[t];
        g.tval[o + t] = val[t];
      }
    }
    if (lane == 0) g.cnt[i] = u2;
    __syncwarp();
  }
}


// Medium rows, staged: one warp per row with at most kStageCap candidates and kStageA entries in A's
// row.  The row's A entries (value, B row start, candidate offset) and then all of its candidates
// (column, B value) are first copied into shared memory with every load of a phase issued at once,
// so the accumulation loop that follows (in ascending A order, as in k_spgemm_warp) touches only
// shared memory instead of waiting on three dependent global loads per A entry.  Other rows go on
// to `next_rows`.
constexpr int kStageCap = 256;
constexpr int kStageA = 64;
constexpr int kStageWarps = 8;

struct WarpStage {
  double cb[kStageCap];
  double hval[kStageCap];
  double ea[kStageA];
  int cj[kStageCap];
  int hkey[kStageCap];
  int epre[kStageA + 1];
  int eb[kStageA];
};

__global__ void __launch_bounds__(kStageWarps * 32) k_spgemm_warp_staged(SpgArgs g, const int* __restrict__ rows,
                                                                         const int* __restrict__ nrows_dev,
                                                                         int* next_rows, int* n_next) {
  extern __shared__ __align__(16) unsigned char stage_raw[];
  constexpr unsigned FULL = 0xffffffffu;
  const int nrows = *nrows_dev;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpStage& W = reinterpret_cast<WarpStage*>(stage_raw)[wid];
  int* key = W.hkey;
  double* val = W.hval;
  const long long gw = (long long)blockIdx.x * kStageWarps + wid;
  const long long nw = (long long)gridDim.x * kStageWarps;
  for (long long ii = gw; ii < nrows; ii += nw) {
    const int i = rows[ii];
    const int ub = (int)(g.ubo[i + 1] - g.ubo[i]);
    const int ab = g.arp[i], na = g.arp[i + 1] - ab;
    if (ub > kStageCap || na > kStageA) {
      if (lane == 0) next_rows[atomicAdd(n_next, 1)] = i;
      continue;
    }
    // A entries: value, B row start, candidate offset (exclusive scan of the B row lengths)
    int carry = 0;
    for (int e0 = 0; e0 < na; e0 += 32) {
      const int e = e0 + lane;
      int len = 0;
      if (e < na) {
        const int l = g.aci[ab + e];
        W.ea[e] = g.av[ab + e];
        int b0, b1;
        spg_brow(g, l, b0, b1);
        W.eb[e] = b0;
        len = b1 - b0;
      }
      int inc = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t;
      }
      if (e < na) W.epre[e] = carry + inc - len;
      carry += __shfl_sync(FULL, inc, 31);
    }
    if (lane == 0) W.epre[na] = carry;
    int H = 32, lg = 5;
    while (H < ub) { H <<= 1; ++lg; }
    for (int t = lane; t < H; t += 32) { key[t] = -1; val[t] = 0.0; }
    __syncwarp();
    // candidates: candidate c belongs to the last A entry whose offset is <= c
    for (int c = lane; c < ub; c += 32) {
      int lo = 0, hi = na - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (W.epre[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      const int q = W.eb[lo] + (c - W.epre[lo]);
      W.cj[c] = g.bci[q];
      W.cb[c] = g.bv[q];
    }
    __syncwarp();
    // accumulate in ascending A order (one A entry at a time, its candidates across the lanes)
    for (int e = 0; e < na; ++e) {
      const int c1 = W.epre[e + 1];
      const double a = W.ea[e];
      for (int c = W.epre[e] + lane; c < c1; c += 32) {
        const int j = W.cj[c];
        unsigned h = ((unsigned)j * 0x9E3779B1u) >> (32 - lg);
        while (true) {
          const int prev = atomicCAS(&key[h], -1, j);
          if (prev == -1 || prev == j) break;
          h = (h + 1) & (H - 1);
        }
        val[h] = fma(a, W.cb[c], val[h]);
      }
      __syncwarp();
    }
    // compact occupied slots to the front (chunks read before written)
    int u = 0;
    for (int base = 0; base < H; base += 32) {
      const int idx = base + lane;
      const int kk = key[idx];
      const double vv = val[idx];
      const bool occ = kk >= 0;
      const unsigned bal = __ballot_sync(FULL, occ);
      __syncwarp();
      if (occ) {
        const int d = u + __popc(bal & ((1u << lane) - 1u));
        key[d] = kk;
        val[d] = vv;
      }
      u += __popc(bal);
      __syncwarp();
    }
    long long mx = 0;
    for (int t = lane; t < u; t += 32) {
      const double c = spg_scale(g, val[t]);
      val[t] = c;
      mx = max(mx, abs_bits(c));
    }
    for (int s2 = 16; s2 > 0; s2 >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, s2));
    const long long thr = spg_thr(g, mx);
    const long long o = g.ubo[i];
    // drop first (the threshold is known), so that only the kept entries are ranked: the ranking
    // costs each lane one pass over the entries per NE of its own
    int u2 = 0;
    for (int base = 0; base < u; base += 32) {
      const int t = base + lane;
      int j = 0;
      double c = 0.0;
      bool keep = false;
      if (t < u) {
        j = key[t];
        c = val[t];
        keep = abs_bits(c) >= thr || (g.keep_diag && j == i);
      }
      const unsigned bal = __ballot_sync(FULL, keep);
      __syncwarp();
      if (keep) {
        const int d = u2 + __popc(bal & ((1u << lane) - 1u));
        key[d] = j;
        val[d] = c;
      }
      u2 += __popc(bal);
      __syncwarp();
    }
    // order by rank among the kept columns (threshold 0: every entry left is kept)
    if (u2 <= 32) spg_rank_write<1>(g, key, val, u2, 0, i, o, lane);
    else if (u2 <= 64) spg_rank_write<2>(g, key, val, u2, 0, i, o, lane);
    else if (u2 <= 128) spg_rank_write<4>(g, key, val, u2, 0, i, o, lane);
    else spg_rank_write<8>(g, key, val, u2, 0, i, o, lane);
    if (lane == 0) g.cnt[i] = u2;
    __syncwarp();
  }
}

// Long rows: one 256-thread CTA per row (grid-stride over the device-side list), dynamic shared
// memory of `cap` ints; a row beyond `cap` candidates sets *err and is skipped.
__global__ void __launch_bounds__(256) k_spgemm_block(SpgArgs g, const int* __restrict__ rows,
                                                      const int* __restrict__ nrows_dev, int cap, int* err) {
  extern __shared__ int bbuf[];
  __shared__ int wcnt[8];
  __shared__ long long wmx[8];
  const int nrows = *nrows_dev;
  for (int rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
  const int i = rows[rr];
  const int t0 = threadIdx.x, lane = t0 & 31, wid = t0 >> 5;
  const long long ub = g.ubo[i + 1] - g.ubo[i];
  if (ub > cap) {
    if (t0 == 0) { atomicOr(err, 1); g.cnt[i] = 0; }
    continue;
  }
  const int ab = g.arp[i], ae = g.arp[i + 1];
  int off = 0;
  for (int k = ab; k < ae; ++k) {
    const int l = g.aci[k];
    int b0, b1;
    spg_brow(g, l, b0, b1);
    const int len = b1 - b0;
    for (int t = t0; t < len; t += 256) bbuf[off + t] = g.bci[b0 + t];
    off += len;
  }
  int P = 256;
  while (P < ub) P <<= 1;
  for (int t = (int)ub + t0; t < P; t += 256) bbuf[t] = 0x7fffffff;
  __syncthreads();
  bitonic_sort<256>(bbuf, P, t0);
  // unique via block-wide chunked compaction (chunk fully read before it is written)
  __shared__ int prev_last;
  if (t0 == 0) prev_last = -1;
  __syncthreads();
  int u = 0;
  for (int base = 0; base < P; base += 256) {
    const int idx = base + t0;
    const int val = bbuf[idx];
    const int prv = (t0 == 0) ? prev_last : bbuf[idx - 1];
    const bool kf = val != 0x7fffffff && val != prv;
    const unsigned bal = __ballot_sync(0xffffffffu, kf);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0, chunk = 0;
    for (int q = 0; q < 8; ++q) { if (q < wid) before += wcnt[q]; chunk += wcnt[q]; }
    if (kf) bbuf[u + before + __popc(bal & ((1u << lane) - 1u))] = val;
    u += chunk;
    if (t0 == 255) prev_last = val;
    __syncthreads();
  }
  const long long o = g.ubo[i];
  long long mx = 0;
  for (int t = t0; t < u; t += 256) {
    const int j = bbuf[t];
    const double c = spg_value(g, ab, ae, j);
    g.tcol[o + t] = j;
    g.tval[o + t] = c;
    mx = max(mx, abs_bits(c));
  }
  for (int s2 = 16; s2 > 0; s2 >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, s2));
  if (lane == 0) wmx[wid] = mx;
  __syncthreads();
  mx = 0;
  for (int q = 0; q < 8; ++q) mx = max(mx, wmx[q]);
  const long long thr = spg_thr(g, mx);
  int outc = 0;
  for (int base = 0; base < u; base += 256) {
    const int t = base + t0;
    int j = 0;
    double c = 0.0;
    bool keep = false;
    if (t < u) {
      j = g.tcol[o + t];
      c = g.tval[o + t];
      keep = abs_bits(c) >= thr || (g.keep_diag && j == i);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wcnt[wid] = __popc(bal);
    __syncthreads();
    int before = 0, chunk = 0;
    for (int q = 0; q < 8; ++q) { if (q < wid) before += wcnt[q]; chunk += wcnt[q]; }
    if (keep) {
      const int d = outc + before + __popc(bal & ((1u << lane) - 1u));
      g.tcol[o + d] = j;
      g.tval[o + d] = c;
    }
    outc += chunk;
    __syncthreads();
  }
  if (t0 == 0) g.cnt[i] = outc;
  __syncthreads();
  }
}

// Block-wide exclusive scan of one int per thread (256 threads); *total receives the sum.
__device__ __forceinline__ int esc_block_scan(int v, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  int before = 0, all = 0;
  for (int q = 0; q < 8; ++q) {
    if (q < wid) before += wsum[q];
    all += wsum[q];
  }
  __syncthreads();
  *total = all;
  return before + inc - v;
}

// Long rows (2048 < candidates <= kEscCap): one 256-thread CTA per row, expand - sort -
// compress.  Every candidate (column j, A entry e, B value) gets a slot in the order A entries
// ascending, each B row ascending; the 64-bit keys j << 32 | slot are sorted (bitonic, in shared
// memory), so each column's candidates sit together in arrival order, and one thread folds each
// run with fma from zero: per output the same ascending-l chain as every other path, hence the
// same bits.  The scaled outputs are dropped against the row's threshold and written in column
// order.  Rows with more candidates or A entries than the shared arrays hold go to `rest_rows`
// (the per-column block kernel).
template <int kEscCap>
constexpr size_t esc_smem() { return (size_t)kEscCap * (8 + 8 + 4 + 4 + 8) + (size_t)(kEscCap / 2 + 1) * 4; }

template <int kEscCap>
__global__ void __launch_bounds__(256) k_spgemm_esc(SpgArgs g, const int* __restrict__ rows,
                                                    const int* __restrict__ nrows_dev, int* rest_rows, int* n_rest) {
  constexpr int kEscMaxA = kEscCap / 2;
  extern __shared__ __align__(16) unsigned char esm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(esm);
  double* bvs = reinterpret_cast<double*>(key + kEscCap);
  double* oval = bvs + kEscCap;
  int* kid = reinterpret_cast<int*>(oval + kEscCap);
  int* ocol = kid + kEscCap;
  int* start = ocol + kEscCap;
  __shared__ int wsum[8];
  __shared__ long long wmx[8];
  const int t0 = threadIdx.x, lane = t0 & 31, wid = t0 >> 5;
  const int nrows = *nrows_dev;
  for (int rr = blockIdx.x; rr < nrows; rr += gridDim.x) {
    const int i = rows[rr];
    const long long ub = g.ubo[i + 1] - g.ubo[i];
    const int ab = g.arp[i], ae = g.arp[i + 1], na = ae - ab;
    if (ub > kEscCap || na > kEscMaxA) {
      if (t0 == 0) rest_rows[atomicAdd(n_rest, 1)] = i;
      continue;
    }
    // slot offsets of the A entries: exclusive scan of their B row lengths
    int carry = 0;
    for (int base = 0; base < na; base += 256) {
      const int e = base + t0;
      int len = 0;
      if (e < na) {
        int b0, b1;
        spg_brow(g, g.aci[ab + e], b0, b1);
        len = b1 - b0;
      }
      int tot;
      const int ex = esc_block_scan(len, wsum, &tot);
      if (e < na) start[e] = carry + ex;
      carry += tot;
    }
    if (t0 == 0) start[na] = carry;
    int P = 256;
    while (P < ub) P <<= 1;
    __syncthreads();
    // expansion: slot s belongs to the last A entry whose start is <= s
    for (int sl = t0; sl < P; sl += 256) {
      if (sl < ub) {
        int lo = 0, hi = na - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (start[mid] <= sl) lo = mid;
          else hi = mid - 1;
        }
        int b0, b1;
        spg_brow(g, g.aci[ab + lo], b0, b1);
        const int q = b0 + (sl - start[lo]);
        key[sl] = ((unsigned long long)(unsigned)g.bci[q] << 32) | (unsigned)sl;
        bvs[sl] = g.bv[q];
        kid[sl] = lo;
      } else {
        key[sl] = ~0ull;
      }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int idx = t0; idx < P; idx += 256) {
          const int ixj = idx ^ j;
          if (ixj > idx) {
            const unsigned long long x = key[idx], y = key[ixj];
            if ((x > y) == ((idx & k) == 0)) {
              key[idx] = y;
              key[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    // runs of one column -> outputs, numbered in column order
    int nout = 0;
    long long mx = 0;
    for (int base = 0; base < (int)ub; base += 256) {
      const int p = base + t0;
      bool head = false;
      if (p < ub) head = (p == 0) || ((key[p] >> 32) != (key[p - 1] >> 32));
      int tot;
      const int oi = nout + esc_block_scan(head ? 1 : 0, wsum, &tot);
      if (head) {
        const unsigned long long jj = key[p] >> 32;
        double acc = 0.0;
        for (int pp = p; pp < ub && (key[pp] >> 32) == jj; ++pp) {
          const int sl = (int)(key[pp] & 0xffffffffu);
          acc = fma(g.av[ab + kid[sl]], bvs[sl], acc);
        }
        const double c = spg_scale(g, acc);
        ocol[oi] = (int)jj;
        oval[oi] = c;
        mx = max(mx, abs_bits(c));
      }
      nout += tot;
    }
    for (int o2 = 16; o2 > 0; o2 >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    if (lane == 0) wmx[wid] = mx;
    __syncthreads();
    mx = 0;
    for (int q = 0; q < 8; ++q) mx = max(mx, wmx[q]);
    const long long thr = spg_thr(g, mx);
    const long long o = g.ubo[i];
    int outc = 0;
    for (int base = 0; base < nout; base += 256) {
      const int t = base + t0;
      bool keep = false;
      int j = 0;
      double c = 0.0;
      if (t < nout) {
        j = ocol[t];
        c = oval[t];
        keep = abs_bits(c) >= thr || (g.keep_diag && j == i);
      }
      int tot;
      const int d = outc + esc_block_scan(keep ? 1 : 0, wsum, &tot);
      if (keep) {
        g.tcol[o + d] = j;
        g.tval[o + d] = c;
      }
      outc += tot;
    }
    if (t0 == 0) g.cnt[i] = outc;
    __syncthreads();
  }
}

// Compaction of the per-row results (at the candidate offsets ubo) into CSR: a CTA takes 256
// consecutive rows, whose output is one contiguous range; each thread finds its entry's row by
// binary search over the CTA's row starts in shared memory, so the writes are coalesced.
__global__ void __launch_bounds__(256) k_spgemm_copy(int ar, const long long* __restrict__ ubo,
                                                     const int* __restrict__ tcol, const double* __restrict__ tval,
                                                     const int* __restrict__ rp, int* __restrict__ ci,
                                                     double* __restrict__ v) {
  __shared__ int srp[257];
  __shared__ long long sub[256];
  const int r0 = blockIdx.x * 256;
  const int nr = min(256, ar - r0);
  for (int t = threadIdx.x; t <= nr; t += 256) srp[t] = rp[r0 + t];
  if (threadIdx.x < nr) sub[threadIdx.x] = ubo[r0 + threadIdx.x];
  __syncthreads();
  const int b = srp[0], e = srp[nr];
  for (int p = b + threadIdx.x; p < e; p += 256) {
    int lo = 0, hi = nr - 1;  // last row whose start is <= p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (srp[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    const long long src = sub[lo] + (p - srp[lo]);
    ci[p] = tcol[src];
    v[p] = tval[src];
  }
}

__global__ void k_i64_to_i32(int n, const long long* __restrict__ in, int* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (int)in[i];
}

// Product into the padded form: row i's cnt[i] entries at tcol/tval + ubo[i] (ubo = exclusive scan
// of the candidate counts).  B is CSR (Bc) or padded (Bp).
// Dynamic shared-memory limits of the product kernels, set once per process (setups may run
// concurrently on several host threads).
static int spgemm_smem_attributes() {
  static std::once_flag once;
  static int rc = AIRG_OK;
  std::call_once(once, [] {
    int r = cuda_status(cudaFuncSetAttribute(k_spgemm_warp_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(WarpStage) * kStageWarps)));
    if (r == AIRG_OK)
      r = cuda_status(cudaFuncSetAttribute(k_spgemm_esc<4096>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)esc_smem<4096>()));
    if (r == AIRG_OK)
      r = cuda_status(cudaFuncSetAttribute(k_spgemm_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(int) * (size_t)kBlockCapMax)));
    rc = r;
  });
  return rc;
}

int spgemm_padded(const DCsr& A, const DCsr* Bc, const SpgPadded* Bp, double scale, double tol, bool keep_diag,
                  SpgPadded& out, Arena& tmp, cudaStream_t s) {
  const int ar = A.nrows;
  long long* ub;
  AIRG_TRY(tmp.alloc(&ub, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&out.ubo, (size_t)ar + 1));
  if (ar > 0)
    airg::note_launch(), k_spgemm_ub<<<GRID(ar)>>>(ar, A.rp, A.ci, Bc ? Bc->rp : nullptr, Bc ? nullptr : Bp->cnt, ub);
  KERNEL_CHECK();
  long long total = 0;
  AIRG_TRY(scan_i64(ub, out.ubo, ar, tmp, s, &total));
  SpgArgs g{};
  g.ar = ar;
  g.arp = A.rp; g.aci = A.ci; g.av = A.v;
  if (Bc) {
    g.brp = Bc->rp; g.bci = Bc->ci; g.bv = Bc->v;
  } else {
    g.bbeg = Bp->beg; g.blen = Bp->cnt; g.bci = Bp->tcol; g.bv = Bp->tval;
  }
  g.scale = scale; g.tol = tol; g.keep_diag = keep_diag ? 1 : 0;
  g.scale_mode = (scale == 1.0) ? 0 : (scale == -1.0 ? 1 : 2);
  g.ubo = out.ubo;
  AIRG_TRY(tmp.alloc(&g.tcol, (size_t)std::max(total, 1LL)));
  AIRG_TRY(tmp.alloc(&g.tval, (size_t)std::max(total, 1LL)));
  AIRG_TRY(tmp.alloc(&g.cnt, std::max(ar, 1)));
  // row lists of the wider paths; counters: [0] mid, [1] big, [2] long, [3] error, [5] rows past
  // the 512-slot tier, [6] longest, [7] rows past the first expand-sort tier
  int *mid, *big, *big2, *lng, *rest, *rest2, *ctr;
  AIRG_TRY(tmp.alloc(&rest2, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&big2, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&mid, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&big, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&lng, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&rest, std::max(ar, 1)));
  AIRG_TRY(tmp.alloc(&ctr, 8));
  CU_TRY(cudaMemsetAsync(ctr, 0, 8 * sizeof(int), s));
  if (ar > 0) {
    airg::note_launch(), k_spgemm_thread<<<grid_for(ar, 128, 152 * 64), 128, 0, s>>>(g, mid, ctr + 0);
    AIRG_TRY(spgemm_smem_attributes());
    const size_t stage_smem = sizeof(WarpStage) * kStageWarps;
    airg::note_launch(), k_spgemm_warp_staged<<<152 * 3, kStageWarps * 32, stage_smem, s>>>(g, mid, ctr + 0, big, ctr + 1);
    // rows of at most 512 candidates: a 512-slot table, eight warps per CTA and four CTAs per SM
    // (twice the warps of the 1024-slot tier)
    airg::note_launch(), k_spgemm_warp<512, 8><<<152 * 4, 8 * 32, 0, s>>>(g, big, ctr + 1, big2, ctr + 5, 512);
    airg::note_launch(), k_spgemm_warp<kWarpCap, 4><<<152 * 4, 4 * 32, 0, s>>>(g, big2, ctr + 5, lng, ctr + 2, kWarpCap);
    // rows of 1025-2048 candidates: the hash warp kernel with a 2048-slot table (two warps per
    // CTA); 2049-4096: expand-sort-compress; beyond: the per-column block kernel.
    // AIRG_SPGEMM_NO_ESC=1 sends every row above 1024 candidates to the block kernel (same results)
    const char* no_esc_env = getenv("AIRG_SPGEMM_NO_ESC");
    const bool no_esc = no_esc_env && no_esc_env[0] == '1';
    const int* blk_rows = lng;
    const int* blk_n = ctr + 2;
    if (!no_esc) {
      airg::note_launch(), k_spgemm_warp<2048, 2><<<152 * 4, 2 * 32, 0, s>>>(g, lng, ctr + 2, rest2, ctr + 7, 2048);
      airg::note_launch(), k_spgemm_esc<4096><<<152, 256, esc_smem<4096>(), s>>>(g, rest2, ctr + 7, rest, ctr + 6);
      blk_rows = rest;
      blk_n = ctr + 6;
    }
    const size_t smem = sizeof(int) * (size_t)kBlockCapMax;
    airg::note_launch(), k_spgemm_block<<<152, 256, smem, s>>>(g, blk_rows, blk_n, kBlockCapMax, ctr + 3);
    KERNEL_CHECK();
  }
  out.nrows = ar;
  out.ncols = Bc ? Bc->ncols : Bp->ncols;
  out.total = total;
  out.cnt = g.cnt;
  out.tcol = g.tcol;
  out.tval = g.tval;
  out.err = ctr + 3;
  out.beg = nullptr;
  if (total <= 0x7fffffffLL) {  // 32-bit row starts, for use as the B operand of another product
    AIRG_TRY(tmp.alloc(&out.beg, std::max(ar, 1)));
    if (ar > 0) airg::note_launch(), k_i64_to_i32<<<GRID(ar)>>>(ar, out.ubo, out.beg);
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

// Compacts a padded product into CSR owned by `own`.
int spgemm_compact(const SpgPadded& P, DCsr& out, Arena& own, Arena& tmp, cudaStream_t s) {
  const int ar = P.nrows;
  int* rp;
  AIRG_TRY(own.alloc(&rp, (size_t)ar + 1));
  int err = 0;
  CU_TRY(cudaMemcpyAsync(&err, P.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  long long nnz = 0;
  AIRG_TRY(scan_i32(P.cnt, rp, ar, tmp, s, &nnz));  // synchronises: err is valid below
  if (err) return AIRG_ERR_UNSUPPORTED;
  if (nnz > 0x7fffffffLL) return AIRG_ERR_UNSUPPORTED;
  out.nrows = ar;
  out.ncols = P.ncols;
  out.nnz = (int)nnz;
  out.rp = rp;
  AIRG_TRY(own.alloc(&out.ci, (size_t)nnz));
  AIRG_TRY(own.alloc(&out.v, (size_t)nnz));
  if (ar > 0) airg::note_launch(), k_spgemm_copy<<<(ar + 255) / 256, 256, 0, s>>>(ar, P.ubo, P.tcol, P.tval, rp, out.ci, out.v);
  KERNEL_CHECK();
  return AIRG_OK;
}

int spgemm(const DCsr& A, const DCsr& B, double scale, double tol, bool keep_diag, DCsr& out, Arena& own,
           Arena& tmp, cudaStream_t s) {
  SpgPadded P;
  AIRG_TRY(spgemm_padded(A, &B, nullptr, scale, tol, keep_diag, P, tmp, s));
  return spgemm_compact(P, out, own, tmp, s);
}

// ------------------------------------------------------------------------------------------
// Step 10: one-point prolongation.  Each F-point takes the strong C dependency with the largest
// |a_ij| (ties: smallest j), else the largest nonzero C entry of its row, weight 1.
// ------------------------------------------------------------------------------------------
__global__ void k_one_point(int n, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                            const uint8_t* __restrict__ strong, const int8_t* __restrict__ cf,
                            const int* __restrict__ fpos, int* __restrict__ w) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    if (cf[i] != kF) continue;
    int best = -1;
    long long bv = -1;  // |a_ij| as bits
    for (int pass = 0; pass < 2 && best < 0; ++pass)
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        const long long a = abs_bits(v[k]);
        if (j == i || cf[j] != kC || a == 0) continue;
        if (pass == 0 && !strong[k]) continue;
        if (a > bv) { bv = a; best = j; }
      }
    w[fpos[i]] = best >= 0 ? best - fpos[best] : -1;
  }
}

// P (n x n_c, natural rows): C row -> its C index, F row -> w (if any), values 1.
__global__ void k_P_count(int n, const int8_t* __restrict__ cf, const int* __restrict__ fpos, const int* __restrict__ w,
                          int* __restrict__ cnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    cnt[i] = (cf[i] == kF) ? (w[fpos[i]] >= 0) : 1;
}
__global__ void k_P_fill(int n, const int8_t* __restrict__ cf, const int* __restrict__ fpos, const int* __restrict__ w,
                         const int* __restrict__ rp, int* __restrict__ ci, double* __restrict__ v) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    const int c = (cf[i] == kF) ? w[fpos[i]] : i - fpos[i];
    if (c >= 0) { ci[rp[i]] = c; v[rp[i]] = 1.0; }
  }
}
// Approximate ideal P = [W; I] in natural row numbering: an F row is W's row, a C row the unit
// entry of its C index.
__global__ void k_Pw_count(int n, const int8_t* __restrict__ cf, const int* __restrict__ fpos, const int* __restrict__ wrp,
                           int* __restrict__ cnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    cnt[i] = (cf[i] == kF) ? wrp[fpos[i] + 1] - wrp[fpos[i]] : 1;
}
__global__ void k_Pw_fill(int n, const int8_t* __restrict__ cf, const int* __restrict__ fpos, DCsr W,
                          const int* __restrict__ rp, int* __restrict__ ci, double* __restrict__ v) {
  for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n; ii += (long long)gridDim.x * blockDim.x) {
    const int i = (int)ii;
    int o = rp[i];
    if (cf[i] == kF) {
      const int f = fpos[i];
      for (int k = W.rp[f]; k < W.rp[f + 1]; ++k) { ci[o] = W.ci[k]; v[o++] = W.v[k]; }
    } else {
      ci[o] = i - fpos[i];
      v[o] = 1.0;
    }
  }
}
// R = [Z I] in natural column numbering: row c = Z row c (columns Fnat[f]) merged with (Cnat[c], 1).
__global__ void k_R_fill(int nc, const int* __restrict__ zrp, const int* __restrict__ zci, const double* __restrict__ zv,
                         const int* __restrict__ Fnat, const int* __restrict__ Cnat, int* __restrict__ rrp,
                         int* __restrict__ rci, double* __restrict__ rv) {
  for (long long cc = (long long)blockIdx.x * blockDim.x + threadIdx.x; cc < nc; cc += (long long)gridDim.x * blockDim.x) {
    const int c = (int)cc;
    const int b = zrp[c], e = zrp[c + 1];
    int o = b + c;
    rrp[c] = o;
    if (c == nc - 1) rrp[nc] = e + nc;
    const int self = Cnat[c];
    bool placed = false;
    for (int k = b; k < e; ++k) {
      const int j = Fnat[zci[k]];
      if (!placed && self < j) { rci[o] = self; rv[o++] = 1.0; placed = true; }
      rci[o] = j;
      rv[o++] = zv[k];
    }
    if (!placed) { rci[o] = self; rv[o] = 1.0; }
  }
}

int build_level(const DCsr& A, const SetupParams& p, int level, bool force_coarsest, LevelBuild& L,
                DCsr& Ac_out, Arena& own, Arena& tmp, cudaStream_t s, const SideStream* side) {
  const int n = A.nrows;
  L.A = A;
  L.n = n;
  auto mark = [&](int k) {
    if (L.ev[k]) cudaEventRecord(L.ev[k], s);
  };
  mark(0);
  const int m = p.poly_order + 1, mc = p.coarse_poly_order + 1;
  bool coarsest = force_coarsest || n <= p.coarse_size || n < m;
  uint8_t* strong = nullptr;
  if (!coarsest) {
    AIRG_TRY(own.alloc(&L.cf, n));
    AIRG_TRY(tmp.alloc(&strong, std::max(A.nnz, 1)));
    int nf = 0;
    if (level < (int)p.cf_reuse.size() && p.cf_reuse[level])
      AIRG_TRY(reuse_split(A, p, p.cf_reuse[level], L.cf, strong, &nf, tmp, s));
    else
      AIRG_TRY(cf_split(A, p, level, L.cf, strong, &nf, tmp, s));
    if (nf == 0 || nf == n) coarsest = true;
    L.nf = nf;
    L.nc = n - nf;
  }
  mark(1);
  if (coarsest) {
    L.coarsest = true;
    L.nf = 0;
    L.nc = 0;
    L.m = mc;
    AIRG_TRY(own.alloc(&L.alpha, mc));
    AIRG_TRY(own.alloc(&L.fitted_dev, 1));
    AIRG_TRY(poly_fit(A, mc, p.seed, level, L.alpha, L.fitted_dev, tmp, s));
    AIRG_TRY(fixed_sparsity_inverse(A, L.alpha, mc, L.Ainv, own, tmp, s, 1));
    mark(2);
    mark(3);
    mark(4);
    mark(5);
    Ac_out = DCsr{};
    return AIRG_OK;
  }
  const int nf = L.nf, nc = L.nc;
  int *isF, *fpos;
  AIRG_TRY(tmp.alloc(&isF, n));
  AIRG_TRY(tmp.alloc(&fpos, (size_t)n + 1));
  airg::note_launch(), k_isF<<<GRID(n)>>>(n, L.cf, isF);
  AIRG_TRY(scan_i32(isF, fpos, n, tmp, s, nullptr));
  AIRG_TRY(own.alloc(&L.pos, n));
  AIRG_TRY(own.alloc(&L.Fnat, nf));
  AIRG_TRY(own.alloc(&L.Cnat, nc));
  airg::note_launch(), k_cf_maps<<<GRID(n)>>>(n, nf, L.cf, fpos, L.pos, L.Fnat, L.Cnat);
  int *cFF, *cFC, *cCF;
  AIRG_TRY(tmp.alloc(&cFF, nf));
  AIRG_TRY(tmp.alloc(&cFC, nf));
  AIRG_TRY(tmp.alloc(&cCF, nc));
  airg::note_launch(), k_extract_count<<<GRID(n)>>>(n, A.rp, A.ci, L.cf, fpos, cFF, cFC, cCF);
  KERNEL_CHECK();
  L.Aff.nrows = nf; L.Aff.ncols = nf;
  L.Afc.nrows = nf; L.Afc.ncols = nc;
  L.Acf.nrows = nc; L.Acf.ncols = nf;
  AIRG_TRY(own.alloc(&L.Aff.rp, (size_t)nf + 1));
  AIRG_TRY(own.alloc(&L.Afc.rp, (size_t)nf + 1));
  AIRG_TRY(own.alloc(&L.Acf.rp, (size_t)nc + 1));
  AIRG_TRY(scan_i32(cFF, L.Aff.rp, nf, tmp, s, nullptr));
  AIRG_TRY(scan_i32(cFC, L.Afc.rp, nf, tmp, s, nullptr));
  AIRG_TRY(scan_i32(cCF, L.Acf.rp, nc, tmp, s, nullptr));
  int tot[3];
  CU_TRY(cudaMemcpyAsync(tot + 0, L.Aff.rp + nf, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaMemcpyAsync(tot + 1, L.Afc.rp + nf, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaMemcpyAsync(tot + 2, L.Acf.rp + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaStreamSynchronize(s));
  const long long zff = tot[0], zfc = tot[1], zcf = tot[2];
  L.Aff.nnz = (int)zff; L.Afc.nnz = (int)zfc; L.Acf.nnz = (int)zcf;
  AIRG_TRY(own.alloc(&L.Aff.ci, zff)); AIRG_TRY(own.alloc(&L.Aff.v, zff));
  AIRG_TRY(own.alloc(&L.Afc.ci, zfc)); AIRG_TRY(own.alloc(&L.Afc.v, zfc));
  AIRG_TRY(own.alloc(&L.Acf.ci, zcf)); AIRG_TRY(own.alloc(&L.Acf.v, zcf));
  airg::note_launch(), k_extract_fill<<<GRID(n)>>>(n, A.rp, A.ci, A.v, L.cf, fpos, L.Aff, L.Afc, L.Acf);
  KERNEL_CHECK();
  mark(2);
  // steps 3-8 on s (no host synchronisation inside)
  L.m = m;
  AIRG_TRY(own.alloc(&L.alpha, m));
  AIRG_TRY(own.alloc(&L.fitted_dev, 1));
  AIRG_TRY(poly_fit(L.Aff, m, p.seed, level, L.alpha, L.fitted_dev, tmp, s));
  AIRG_TRY(fixed_sparsity_inverse(L.Aff, L.alpha, m, L.Ainv, own, tmp, s, p.sparsity_order));
  // steps 10-11a (one-point P and A P) need only the splitting: on the side stream, they overlap
  // the polynomial fit
  AIRG_TRY(own.alloc(&L.w, nf));
  cudaStream_t s2 = s;
  Arena* tmp2 = &tmp;
  if (side && side->s) {
    CU_TRY(cudaEventRecord(side->fork, s));
    CU_TRY(cudaStreamWaitEvent(side->s, side->fork, 0));
    s2 = side->s;
    tmp2 = side->tmp;
  }
  airg::note_launch(), k_one_point<<<grid_for(n, 256), 256, 0, s2>>>(n, A.rp, A.ci, A.v, strong, L.cf, fpos, L.w);
  KERNEL_CHECK();
  // A P stays in the padded form of the product (no compaction): R reads its rows in place
  SpgPadded AP;
  if (!p.ideal_prolong) {
    DCsr P;
    P.nrows = n; P.ncols = nc;
    int* pc;
    AIRG_TRY(tmp2->alloc(&pc, n));
    AIRG_TRY(tmp2->alloc(&P.rp, (size_t)n + 1));
    airg::note_launch(), k_P_count<<<grid_for(n, 256), 256, 0, s2>>>(n, L.cf, fpos, L.w, pc);
    AIRG_TRY(scan_i32(pc, P.rp, n, *tmp2, s2, nullptr));
    P.nnz = n;  // upper bound (only P.rp delimits rows); avoids a synchronisation
    AIRG_TRY(tmp2->alloc(&P.ci, n));
    AIRG_TRY(tmp2->alloc(&P.v, n));
    airg::note_launch(), k_P_fill<<<grid_for(n, 256), 256, 0, s2>>>(n, L.cf, fpos, L.w, P.rp, P.ci, P.v);
    KERNEL_CHECK();
    AIRG_TRY(spgemm_padded(A, &P, nullptr, 1.0, 0.0, false, AP, *tmp2, s2));
  }
  if (s2 != s) CU_TRY(cudaEventRecord(side->join, s2));
  mark(3);
  // step 9
  AIRG_TRY(spgemm(L.Acf, L.Ainv, -1.0, p.drop_R, false, L.Z, own, tmp, s));
  mark(4);
  // step 10's alternative (eq. prolong): W = -Ainv A_fc with Z's drop, then P = [W; I] and A P
  if (p.ideal_prolong) {
    AIRG_TRY(spgemm(L.Ainv, L.Afc, -1.0, p.drop_R, false, L.W, own, tmp, s));
    DCsr P;
    P.nrows = n; P.ncols = nc; P.nnz = L.W.nnz + nc;
    int* pc;
    AIRG_TRY(tmp.alloc(&pc, n));
    AIRG_TRY(tmp.alloc(&P.rp, (size_t)n + 1));
    AIRG_TRY(tmp.alloc(&P.ci, std::max(P.nnz, 1)));
    AIRG_TRY(tmp.alloc(&P.v, std::max(P.nnz, 1)));
    airg::note_launch(), k_Pw_count<<<grid_for(n, 256), 256, 0, s>>>(n, L.cf, fpos, L.W.rp, pc);
    AIRG_TRY(scan_i32(pc, P.rp, n, tmp, s, nullptr));
    airg::note_launch(), k_Pw_fill<<<grid_for(n, 256), 256, 0, s>>>(n, L.cf, fpos, L.W, P.rp, P.ci, P.v);
    KERNEL_CHECK();
    AIRG_TRY(spgemm_padded(A, &P, nullptr, 1.0, 0.0, false, AP, tmp, s));
  }
  // step 11b: A_c = R (A P)
  DCsr R;
  R.nrows = nc; R.ncols = n; R.nnz = L.Z.nnz + nc;
  AIRG_TRY(tmp.alloc(&R.rp, (size_t)nc + 1));
  AIRG_TRY(tmp.alloc(&R.ci, R.nnz));
  AIRG_TRY(tmp.alloc(&R.v, R.nnz));
  if (nc > 0) airg::note_launch(), k_R_fill<<<GRID(nc)>>>(nc, L.Z.rp, L.Z.ci, L.Z.v, L.Fnat, L.Cnat, R.rp, R.ci, R.v);
  KERNEL_CHECK();
  if (s2 != s) CU_TRY(cudaStreamWaitEvent(s, side->join, 0));
  if (AP.beg) {
    SpgPadded RAP;
    AIRG_TRY(spgemm_padded(R, nullptr, &AP, 1.0, p.drop_Ac, true, RAP, tmp, s));
    int ap_err = 0;
    CU_TRY(cudaMemcpyAsync(&ap_err, AP.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    AIRG_TRY(spgemm_compact(RAP, Ac_out, own, tmp, s));  // synchronises: ap_err is valid below
    if (ap_err) return AIRG_ERR_UNSUPPORTED;
  } else {
    DCsr APc;
    AIRG_TRY(spgemm_compact(AP, APc, tmp, tmp, s));
    AIRG_TRY(spgemm(R, APc, 1.0, p.drop_Ac, true, Ac_out, own, tmp, s));
  }
  mark(5);
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Solve-phase operators in the F-then-C numbering
// ------------------------------------------------------------------------------------------
// Last row of the block's window [0, nr) whose start is <= p (empty rows share their successor's
// start, so the row found is the one that holds entry p).
__device__ __forceinline__ int window_row(const int* srp, int nr, int p) {
  int lo = 0, hi = nr - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (srp[mid] <= p) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// AF row f = A_ff row f, then A_fc row f with columns nf + pos_next[c].  Entry-parallel: a block
// takes 256 rows, stages both row-pointer windows in shared memory, and each thread moves single
// entries (an A_ff entry p of row f goes to p + Afc.rp[f], an A_fc entry to p + Aff.rp[f + 1]), so
// loads and stores are coalesced instead of each thread walking its own short row.
__global__ void __launch_bounds__(256) k_af_fill(int nf, DCsr Aff, DCsr Afc, const int* __restrict__ pos_next, DCsr AF) {
  __shared__ int sff[257], sfc[257];
  const int r0 = blockIdx.x * 256;
  const int nr = min(256, nf - r0);
  for (int t = threadIdx.x; t <= nr; t += 256) {
    sff[t] = Aff.rp[r0 + t];
    sfc[t] = Afc.rp[r0 + t];
  }
  __syncthreads();
  if ((int)threadIdx.x < nr) AF.rp[r0 + threadIdx.x] = sff[threadIdx.x] + sfc[threadIdx.x];
  if (threadIdx.x == 0 && r0 + nr == nf) AF.rp[nf] = sff[nr] + sfc[nr];
  for (int p = sff[0] + threadIdx.x; p < sff[nr]; p += 256) {
    const int o = p + sfc[window_row(sff, nr, p)];
    AF.ci[o] = Aff.ci[p];
    AF.v[o] = Aff.v[p];
  }
  for (int p = sfc[0] + threadIdx.x; p < sfc[nr]; p += 256) {
    const int o = p + sff[window_row(sfc, nr, p) + 1];
    const int c = Afc.ci[p];
    AF.ci[o] = nf + (pos_next ? pos_next[c] : c);
    AF.v[o] = Afc.v[p];
  }
}
__global__ void k_perm_rows_count(int n, const int* __restrict__ rp, const int* __restrict__ pos, int* __restrict__ cnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    cnt[pos ? pos[i] : i] = rp[i + 1] - rp[i];
}
// row pos[i] of out <- row i of A; columns mapped by cpos (nullptr: kept).  Entry-parallel over the
// source rows (a block takes 256 of them with their source and destination row starts in shared
// memory), so the reads are coalesced and each row's writes stay contiguous.
__global__ void __launch_bounds__(256) k_perm_rows_fill(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                        const double* __restrict__ v, const int* __restrict__ pos,
                                                        const int* __restrict__ cpos, const int* __restrict__ orp,
                                                        int* __restrict__ oci, double* __restrict__ ov) {
  __shared__ int srp[257], sdst[256];
  const int r0 = blockIdx.x * 256;
  const int nr = min(256, n - r0);
  for (int t = threadIdx.x; t <= nr; t += 256) srp[t] = rp[r0 + t];
  if ((int)threadIdx.x < nr) {
    const int i = r0 + threadIdx.x;
    sdst[threadIdx.x] = orp[pos ? pos[i] : i];
  }
  __syncthreads();
  for (int p = srp[0] + threadIdx.x; p < srp[nr]; p += 256) {
    const int lo = window_row(srp, nr, p);
    const int o = sdst[lo] + (p - srp[lo]);
    const int j = ci[p];
    oci[o] = cpos ? cpos[j] : j;
    ov[o] = v[p];
  }
}
__global__ void k_w_solve(int nf, const int* __restrict__ w, const int* __restrict__ pos_next, int* __restrict__ ws) {
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    const int c = w[f];
    ws[f] = c < 0 ? -1 : (pos_next ? pos_next[c] : c);
  }
}

// Nested solve numbering of a level: F-points first (ascending), then the C-points in the next
// level's own nested numbering.  lay(i) = pos(i) for F, n_f + lay_next(pos(i) - n_f) for C.
__global__ void k_compose_layout(int n, int nf, const int* __restrict__ pos, const int* __restrict__ lay_next,
                                 int* __restrict__ lay) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int p = pos[i];
    lay[i] = (p < nf || !lay_next) ? p : nf + lay_next[p - nf];
  }
}

int compose_layout(const LevelBuild& L, const int* lay_next, int* lay, cudaStream_t s) {
  if (L.n > 0) airg::note_launch(), k_compose_layout<<<GRID(L.n)>>>(L.n, L.nf, L.pos, lay_next, lay);
  KERNEL_CHECK();
  return AIRG_OK;
}

int build_solve_ops(const LevelBuild& L, const int* pos_next, DCsr& AF, DCsr& Zs, int** ws, DCsr& Ws, Arena& own,
                    Arena& tmp, cudaStream_t s) {
  const int nf = L.nf, nc = L.nc;
  AIRG_TRY(own.csr(AF, nf, nf + nc, L.Aff.nnz + L.Afc.nnz));
  if (nf > 0) airg::note_launch(), k_af_fill<<<ceil_div(nf, 256), 256, 0, s>>>(nf, L.Aff, L.Afc, pos_next, AF);
  KERNEL_CHECK();
  AIRG_TRY(own.csr(Zs, nc, nf, L.Z.nnz));
  int* cnt;
  AIRG_TRY(tmp.alloc(&cnt, std::max(nc, 1)));
  if (nc > 0) airg::note_launch(), k_perm_rows_count<<<GRID(nc)>>>(nc, L.Z.rp, pos_next, cnt);
  AIRG_TRY(scan_i32(cnt, Zs.rp, nc, tmp, s, nullptr));
  if (nc > 0)
    airg::note_launch(), k_perm_rows_fill<<<ceil_div(nc, 256), 256, 0, s>>>(nc, L.Z.rp, L.Z.ci, L.Z.v, pos_next, nullptr,
                                                                           Zs.rp, Zs.ci, Zs.v);
  AIRG_TRY(own.alloc(ws, std::max(nf, 1)));
  if (nf > 0) airg::note_launch(), k_w_solve<<<GRID(nf)>>>(nf, L.w, pos_next, *ws);
  KERNEL_CHECK();
  // approximate ideal W: the same rows, columns in the next level's numbering
  if (L.W.nrows > 0) {
    AIRG_TRY(own.csr(Ws, nf, nc, L.W.nnz));
    int* wcnt;
    AIRG_TRY(tmp.alloc(&wcnt, std::max(nf, 1)));
    airg::note_launch(), k_perm_rows_count<<<GRID(nf)>>>(nf, L.W.rp, nullptr, wcnt);
    AIRG_TRY(scan_i32(wcnt, Ws.rp, nf, tmp, s, nullptr));
    airg::note_launch(), k_perm_rows_fill<<<ceil_div(nf, 256), 256, 0, s>>>(nf, L.W.rp, L.W.ci, L.W.v, nullptr, pos_next,
                                                                           Ws.rp, Ws.ci, Ws.v);
    KERNEL_CHECK();
  }
  return AIRG_OK;
}

int permute_matrix(const DCsr& A, const int* pos, DCsr& out, Arena& own, Arena& tmp, cudaStream_t s) {
  const int n = A.nrows;
  AIRG_TRY(own.csr(out, n, n, A.nnz));
  int* cnt;
  AIRG_TRY(tmp.alloc(&cnt, std::max(n, 1)));
  if (n > 0) airg::note_launch(), k_perm_rows_count<<<GRID(n)>>>(n, A.rp, pos, cnt);
  AIRG_TRY(scan_i32(cnt, out.rp, n, tmp, s, nullptr));
  if (n > 0)
    airg::note_launch(), k_perm_rows_fill<<<ceil_div(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, pos, pos, out.rp, out.ci,
                                                                          out.v);
  KERNEL_CHECK();
  return AIRG_OK;
}

}  // namespace airg
