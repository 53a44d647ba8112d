// Primitive kernels: scans, deterministic FP64 reductions, CSR SpMV with fused epilogues,
// Gram-Schmidt passes and small vector kernels.  All of them are bandwidth-bound; none uses tensor
// cores (nothing here is a dense contraction).
#include <cuda_bf16.h>

#include <cstdlib>

#include "airg_common.cuh"

namespace airg {

// ------------------------------------------------------------------------------------------
// Block-level helpers
// ------------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Exclusive scan across a block of blockDim.x (multiple of 32, <= 1024) threads.
template <class T>
__device__ T block_excl_scan(T v, T* total) {
  __shared__ T wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T t = lane < nw ? wsum[lane] : T(0);
    T ti = warp_incl_scan(t);
    if (lane < nw) wsum[lane] = ti - t;
    if (lane == nw - 1 && total) *total = ti;
  }
  __syncthreads();
  T r = inc - v + wsum[wid];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------------------------------
// Exclusive scan (three kernels: tile sums, recursive scan of tile sums, tile scans)
// ------------------------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__global__ void k_tile_sum(const T* __restrict__ in, T* __restrict__ tsum, int n) {
  long long base = (long long)blockIdx.x * kScanTile;
  T s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
    long long g = base + i;
    if (g < n) s += in[g];
  }
  __shared__ T tot;
  T ex = block_excl_scan<T>(s, &tot);
  (void)ex;
  __syncthreads();
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

template <class T>
__global__ void k_tile_scan(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ toff, int n) {
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  T v[kScanItems];
  T loc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    long long g = base + j;
    v[j] = g < n ? in[g] : T(0);
    loc += v[j];
  }
  T run = block_excl_scan<T>(loc, (T*)nullptr) + (toff ? toff[blockIdx.x] : T(0));
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    long long g = base + j;
    if (g < n) out[g] = run;
    run += v[j];
    if (g == n - 1) out[n] = run;
  }
}

// One CTA scans up to kScanSingle entries in one launch (tiles of 1024 x 8 in sequence, carrying
// the running offset): on small levels the launch count, not the bandwidth, is what costs.
constexpr int kScanSingle = 1 << 16;

template <class T>
__global__ void __launch_bounds__(1024) k_scan_single(const T* __restrict__ in, T* __restrict__ out, int n) {
  __shared__ T carry, tot;
  if (threadIdx.x == 0) carry = T(0);
  __syncthreads();
  for (int base = 0; base < n; base += 1024 * kScanItems) {
    const int b0 = base + threadIdx.x * kScanItems;
    T v[kScanItems];
    T loc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      v[j] = (b0 + j < n) ? in[b0 + j] : T(0);
      loc += v[j];
    }
    T run = block_excl_scan<T>(loc, &tot) + carry;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
      if (b0 + j < n) out[b0 + j] = run;
      run += v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

template <class T>
static int scan_impl(const T* in, T* out, int n, Arena& tmp, cudaStream_t s, long long* total_host) {
  if (n <= 0) {
    CU_TRY(cudaMemsetAsync(out, 0, sizeof(T), s));
    if (total_host) *total_host = 0;
    return AIRG_OK;
  }
  int nt = ceil_div(n, kScanTile);
  T* toff = nullptr;
  if (nt > 1 && n <= kScanSingle) {
    airg::note_launch(), k_scan_single<T><<<1, 1024, 0, s>>>(in, out, n);
    KERNEL_CHECK();
    nt = 0;
  } else if (nt > 1) {
    T* tsum = nullptr;
    AIRG_TRY(tmp.alloc(&tsum, nt));
    AIRG_TRY(tmp.alloc(&toff, (size_t)nt + 1));
    airg::note_launch(), k_tile_sum<T><<<nt, kScanThreads, 0, s>>>(in, tsum, n);
    KERNEL_CHECK();
    AIRG_TRY(scan_impl<T>(tsum, toff, nt, tmp, s, nullptr));
  }
  if (nt > 0) {
    airg::note_launch(), k_tile_scan<T><<<nt, kScanThreads, 0, s>>>(in, out, toff, n);
    KERNEL_CHECK();
  }
  if (total_host) {
    T t = 0;
    CU_TRY(cudaMemcpyAsync(&t, out + n, sizeof(T), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    *total_host = (long long)t;
  }
  return AIRG_OK;
}

int scan_i32(const int* in, int* out, int n, Arena& tmp, cudaStream_t s, long long* total_host) {
  return scan_impl<int>(in, out, n, tmp, s, total_host);
}
int scan_i64(const long long* in, long long* out, int n, Arena& tmp, cudaStream_t s, long long* total_host) {
  return scan_impl<long long>(in, out, n, tmp, s, total_host);
}

// ------------------------------------------------------------------------------------------
// Deterministic reductions
// ------------------------------------------------------------------------------------------
int reducer_init(Reducer& r, Arena& a, cudaStream_t s) {
  AIRG_TRY(a.alloc(&r.partial, (size_t)kRedBlocks * kRedCols));
  AIRG_TRY(a.alloc(&r.counter, 1));
  CU_TRY(cudaMemsetAsync(r.counter, 0, sizeof(unsigned), s));
  return AIRG_OK;
}

// Reduces acc[0..nv) across the block, writes the block's partials, and lets the last block to
// finish sum all partials (in a fixed order) into out[0..nv).  Fixed grid => deterministic.
template <int NV>
__device__ void block_partials_finish(const double (&acc)[NV], int nv, double* partial, unsigned* counter,
                                      double* out0, int nout0, double* out1) {
  __shared__ double red[8][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    if (k < nv) {
      double t = warp_sum(acc[k]);
      if (lane == 0) red[wid][k] = t;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w][k];
    partial[(size_t)blockIdx.x * kRedCols + k] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // one warp per value: lane l sums the partials of blocks l, l+32, ... in order, then a fixed
  // butterfly (short FP64 chains: FP64 latency on sm_103a is tens of clocks per add)
  for (int k = wid; k < nv; k += nw) {
    double t = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) t += ((volatile double*)partial)[(size_t)b * kRedCols + k];
    t = warp_sum(t);
    if (lane == 0) {
      if (k < nout0) {
        if (out0) out0[k] = t;
      } else if (out1) {
        out1[0] = t;
      }
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

__global__ void __launch_bounds__(256) k_nrm2sq(const double* __restrict__ x, int n, double* out,
                                                double* partial, unsigned* counter) {
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double t = x[i];
    acc[0] += t * t;
  }
  block_partials_finish<1>(acc, 1, partial, counter, out, 1, nullptr);
}

int dev_nrm2sq(const double* x, int n, double* out, Reducer& r, cudaStream_t s) {
  airg::note_launch(), k_nrm2sq<<<kRedBlocks, 256, 0, s>>>(x, n, out, r.partial, r.counter);
  KERNEL_CHECK();
  return AIRG_OK;
}

template <int NC>
__global__ void __launch_bounds__(256) k_gs_pass(const double* __restrict__ V, long long ldv, int ncols,
                                                 double* __restrict__ w, int n, const double* __restrict__ hsub,
                                                 double* dots, double* nrm, double* partial, unsigned* counter) {
  (void)ncols;  // == NC
  __shared__ double sh[NC];
  if (hsub)
    for (int k = threadIdx.x; k < NC; k += blockDim.x) sh[k] = hsub[k];
  __syncthreads();
  const bool want = dots != nullptr;  // dot products wanted
  double acc[NC + 1];
#pragma unroll
  for (int k = 0; k <= NC; ++k) acc[k] = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double wr = w[r];
    double vk[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) vk[k] = V[(size_t)k * ldv + r];
    if (hsub) {
      // two interleaved partial sums halve the dependent FP64 chain
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int k = 0; k < NC; k += 2) {
        s0 = fma(vk[k], sh[k], s0);
        if (k + 1 < NC) s1 = fma(vk[k + 1], sh[k + 1], s1);
      }
      wr -= s0 + s1;
      w[r] = wr;
    }
    if (want) {
#pragma unroll
      for (int k = 0; k < NC; ++k) acc[k] = fma(vk[k], wr, acc[k]);
    }
    acc[NC] = fma(wr, wr, acc[NC]);
  }
  // place the norm accumulator right after the dots so one finish call reduces nd+1 values
  const int nd = want ? NC : 0;
  if (!want) acc[0] = acc[NC];
  block_partials_finish<NC + 1>(acc, nd + 1, partial, counter, dots, nd, nrm);
}

// One instance per column count, so no FP64 instruction is spent on absent columns (sm_103a's FP64
// issue rate, not HBM, bounds these passes).
template <int NC>
static void gs_launch(const double* V, long long ldv, int ncols, double* w, int n, const double* hsub, double* dots,
                      double* nrm, Reducer& r, cudaStream_t s) {
  airg::note_launch(), k_gs_pass<NC><<<kRedBlocks, 256, 0, s>>>(V, ldv, ncols, w, n, hsub, dots, nrm, r.partial, r.counter);
}

int dev_gs_pass(const double* V, long long ldv, int ncols, double* w, int n, const double* hsub, double* dots,
                double* nrm, Reducer& r, cudaStream_t s) {
  switch (ncols) {
#define AIRG_GS_CASE(c) \
  case c: gs_launch<c>(V, ldv, ncols, w, n, hsub, dots, nrm, r, s); break;
    AIRG_GS_CASE(1) AIRG_GS_CASE(2) AIRG_GS_CASE(3) AIRG_GS_CASE(4) AIRG_GS_CASE(5) AIRG_GS_CASE(6)
    AIRG_GS_CASE(7) AIRG_GS_CASE(8) AIRG_GS_CASE(9) AIRG_GS_CASE(10) AIRG_GS_CASE(11) AIRG_GS_CASE(12)
    AIRG_GS_CASE(13) AIRG_GS_CASE(14) AIRG_GS_CASE(15) AIRG_GS_CASE(16) AIRG_GS_CASE(17) AIRG_GS_CASE(18)
    AIRG_GS_CASE(19) AIRG_GS_CASE(20) AIRG_GS_CASE(21) AIRG_GS_CASE(22) AIRG_GS_CASE(23) AIRG_GS_CASE(24)
    AIRG_GS_CASE(25) AIRG_GS_CASE(26) AIRG_GS_CASE(27) AIRG_GS_CASE(28) AIRG_GS_CASE(29) AIRG_GS_CASE(30)
    AIRG_GS_CASE(31) AIRG_GS_CASE(32)
#undef AIRG_GS_CASE
    default: return AIRG_ERR_ARG;
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

__global__ void k_multi_axpy(const double* __restrict__ V, long long ldv, int ncols, const double* __restrict__ y,
                             double* __restrict__ x, int n) {
  __shared__ double sy[64];
  for (int k = threadIdx.x; k < ncols; k += blockDim.x) sy[k] = y[k];
  __syncthreads();
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double t = x[r];
    for (int k = 0; k < ncols; ++k) t += sy[k] * V[(size_t)k * ldv + r];
    x[r] = t;
  }
}

int dev_multi_axpy(const double* V, long long ldv, int ncols, const double* y, double* x, int n, cudaStream_t s) {
  if (ncols <= 0) return AIRG_OK;
  if (ncols > 64) return AIRG_ERR_ARG;
  airg::note_launch(), k_multi_axpy<<<grid_for(n, 256), 256, 0, s>>>(V, ldv, ncols, y, x, n);
  KERNEL_CHECK();
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// CSR SpMV.  Every kernel reads the rows' entries directly (columns and values with an L2 policy
// chosen per operator, see l2_policy), gathers x and accumulates with one fused multiply-add
// per entry: one thread per row for short rows (k_spmv_row), LPR lanes per row for longer ones
// (k_spmv_vec).  PROLONG: first F-smoothing residual with the one-point prolongation fused in (see
// dev_spmv_resid_prolong).  VT is the stored value type (double, float or bf16), XT the vector and
// accumulation type (double for the FP64 path, float for the mixed-precision V-cycle).
// ------------------------------------------------------------------------------------------
constexpr int kSpmvThreads = 256;

template <typename VT, typename XT>
__device__ __forceinline__ XT vfma(VT a, XT x, XT acc);
template <>
__device__ __forceinline__ double vfma<double, double>(double a, double x, double acc) { return fma(a, x, acc); }
template <>
__device__ __forceinline__ float vfma<float, float>(float a, float x, float acc) { return fmaf(a, x, acc); }
template <>
__device__ __forceinline__ float vfma<__nv_bfloat16, float>(__nv_bfloat16 a, float x, float acc) {
  return fmaf(__bfloat162float(a), x, acc);
}



// Entries k0, k0 + STRIDE, ..., k0 + (R-1) STRIDE of a row (those below re): loads, then gathers
// of x, then R FMAs in entry order.  R is a compile-time count, so that the FP64 FMAs a warp issues
// stop at its longest row (or lane share): on sm_103a the FP64 pipe takes about 64 cycles per warp
// instruction whether or not its lanes are predicated off, and the SpMVs are close to that pipe's
// rate.
template <typename VT, typename XT, bool PROLONG, int R, int STRIDE = 1>
__device__ __forceinline__ XT row_entries(const int* __restrict__ ci, const VT* __restrict__ v, int k0, int re,
                                          const XT* x, int nrows, const int* __restrict__ w, XT s, uint64_t pol) {
  VT a[R];
  XT xv[R];
  int c[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int k = k0 + t * STRIDE;
    c[t] = (k < re) ? ld_pol(ci + k, pol) : -1;
    a[t] = (k < re) ? ld_pol(v + k, pol) : VT(0);
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    xv[t] = XT(0);
    if (c[t] >= 0) {
      if (PROLONG && c[t] < nrows) {
        const int src = w[c[t]];
        xv[t] = src >= 0 ? x[nrows + src] : XT(0);
      } else {
        xv[t] = __ldg(x + c[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t)
    if (c[t] >= 0) s = vfma<VT, XT>(a[t], xv[t], s);
  return s;
}

// The last r (< RB) entries of a row or lane share, with an exact compile-time count.
template <typename VT, typename XT, bool PROLONG, int RB, int STRIDE>
__device__ __forceinline__ XT entries_tail(int r, const int* __restrict__ ci, const VT* __restrict__ v, int k0, int re,
                                           const XT* x, int nrows, const int* __restrict__ w, XT s, uint64_t pol) {
  switch (r) {
    case 1: return row_entries<VT, XT, PROLONG, 1, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
    case 2: return row_entries<VT, XT, PROLONG, 2, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
    case 3: return row_entries<VT, XT, PROLONG, 3, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
    default: break;
  }
  if constexpr (RB > 4) {
    switch (r) {
      case 4: return row_entries<VT, XT, PROLONG, 4, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
      case 5: return row_entries<VT, XT, PROLONG, 5, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
      case 6: return row_entries<VT, XT, PROLONG, 6, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
      case 7: return row_entries<VT, XT, PROLONG, 7, STRIDE>(ci, v, k0, re, x, nrows, w, s, pol);
      default: break;
    }
  }
  return s;
}

// The row's own operand of the output (b, or y for the accumulating mode), loaded before the
// entries so that its round trip overlaps theirs instead of following the sum.
template <int MODE, typename XT>
__device__ __forceinline__ XT row_operand(const XT* b, const XT* y, int row) {
  if (MODE == SPMV_SET) return XT(0);
  if (MODE == SPMV_ADD) return y[row];
  return b[row];
}
template <int MODE, typename XT>
__device__ __forceinline__ XT row_output(XT pre, XT s, const XT* __restrict__ coef) {
  if (MODE == SPMV_SET) return s;
  if (MODE == SPMV_RESID) return pre - s;
  if (MODE == SPMV_AXPB) return coef[0] * pre + s;
  return pre + s;  // SPMV_ADD, SPMV_ADDB
}
// One-point prolongation of the row's own F-point (PROLONG): its C source's value, or 0.
template <typename XT>
__device__ __forceinline__ XT row_prolong(const XT* x, int nrows, const int* __restrict__ w, int row) {
  const int src = w[row];
  return src >= 0 ? x[nrows + src] : XT(0);
}

// Short rows (average <= 12 entries): one thread per row reads its own entries directly, kRowBatch
// (4 for rows of about 4 entries or fewer, else 8) at a time (the warp's rows are contiguous, so
// the lines they touch arrive once in L1), up to the warp's longest row, and accumulates with one
// fused multiply-add per entry, in storage order; no shared memory and no barrier.  Resident CTAs
// per SM the register budget allows: eight (32 registers) for the 4-entry batches, five (48) for
// the 8-entry ones; the fused-prolongation variants are left unbounded.
constexpr int kRowBlocks4 = 8, kRowBlocks8 = 5;
template <typename VT, typename XT, int MODE, bool PROLONG, int kRowBatch>
__global__ void __launch_bounds__(256, PROLONG ? 1 : (kRowBatch == 4 ? kRowBlocks4 : kRowBlocks8))
    k_spmv_row(int nrows, const int* __restrict__ rp, const int* __restrict__ ci, const VT* __restrict__ v, const XT* x,
               const XT* b, XT* y, const int* __restrict__ w, XT* xf, const XT* __restrict__ coef, bool keep) {
  const uint64_t pol = l2_policy(keep);
  // the grid holds one thread per row
  const long long rr = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (rr < nrows) {
    const int row = (int)rr;
    const XT pre = row_operand<MODE>(b, y, row);
    const XT pro = PROLONG ? row_prolong(x, nrows, w, row) : XT(0);
    const int rb = rp[row], re = rp[row + 1];
    const int wmax = (int)__reduce_max_sync(__activemask(), (unsigned)(re - rb));  // uniform over the lanes here
    XT s = XT(0);
    int j0 = 0;
    for (; j0 + kRowBatch <= wmax; j0 += kRowBatch)
      s = row_entries<VT, XT, PROLONG, kRowBatch>(ci, v, rb + j0, re, x, nrows, w, s, pol);
    s = entries_tail<VT, XT, PROLONG, kRowBatch, 1>(wmax - j0, ci, v, rb + j0, re, x, nrows, w, s, pol);
    y[row] = row_output<MODE>(pre, s, coef);
    if (PROLONG) xf[row] = pro;
  }
}

// Longer rows (LPR = 2..32 lanes per row): the LPR lanes of a row read its entries directly, lane l
// taking entries l, l + LPR, ..., 8 per batch up to the warp's largest lane share (so the warp
// issues exactly that many FMAs and one round trip of loads per batch), accumulate with FMAs and
// combine by a butterfly over the LPR lanes.  No shared memory and no barrier.  Five resident CTAs
// per SM (48 registers); the fused-prolongation variant, whose gathers hold more registers, takes
// 4-entry batches at six CTAs, so that the small levels' launches fit in one wave.
constexpr int kVecBlocks = 5, kVecBlocksProlong = 6;
template <typename VT, typename XT, int LPR, int MODE, bool PROLONG>
__global__ void __launch_bounds__(256, PROLONG ? kVecBlocksProlong : kVecBlocks)
    k_spmv_vec(int nrows, const int* __restrict__ rp, const int* __restrict__ ci, const VT* __restrict__ v, const XT* x,
               const XT* b, XT* y, const int* __restrict__ w, XT* xf, const XT* __restrict__ coef, bool keep) {
  constexpr int GPW = 32 / LPR;  // rows per warp and pass
  constexpr int kVecBatch = PROLONG ? 4 : 8;
  const uint64_t pol = l2_policy(keep);
  const int lane = threadIdx.x % LPR, grp = (threadIdx.x & 31) / LPR;
  // the grid holds one group of LPR lanes per row; the test below is warp-uniform, so that every
  // lane reaches the butterfly
  const long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * GPW;
  if (base < nrows) {
    const long long rr = base + grp;
    const bool act = rr < nrows;
    const int row = act ? (int)rr : 0;
    const bool own = act && lane == 0;
    const XT pre = own ? row_operand<MODE>(b, y, row) : XT(0);
    const XT pro = (PROLONG && own) ? row_prolong(x, nrows, w, row) : XT(0);
    const int rb = act ? rp[row] : 0, re = act ? rp[row + 1] : 0;
    const int mine = re - rb > lane ? (re - rb - lane + LPR - 1) / LPR : 0;  // this lane's entries
    const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)mine);
    const int k0 = rb + lane;
    XT s = XT(0);
    int j0 = 0;
    for (; j0 + kVecBatch <= wmax; j0 += kVecBatch)
      s = row_entries<VT, XT, PROLONG, kVecBatch, LPR>(ci, v, k0 + j0 * LPR, re, x, nrows, w, s, pol);
    s = entries_tail<VT, XT, PROLONG, kVecBatch, LPR>(wmax - j0, ci, v, k0 + j0 * LPR, re, x, nrows, w, s, pol);
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (own) {
      y[row] = row_output<MODE>(pre, s, coef);
      if (PROLONG) xf[row] = pro;
    }
  }
}

template <typename VT, typename XT, int RB>
static void launch_spmv_row(int nrows, const int* rp, const int* ci, const VT* v, const XT* x, const XT* b, XT* y,
                            int mode, const int* w, XT* xf, cudaStream_t s, const XT* coef, bool keep) {
  const int g1 = ceil_div(nrows, 256);
  if (w) {
    airg::note_launch(), k_spmv_row<VT, XT, SPMV_RESID, true, RB><<<g1, 256, 0, s>>>(nrows, rp, ci, v, x, b, y, w, xf, nullptr, keep);
    return;
  }
  switch (mode) {
    case SPMV_SET: airg::note_launch(), k_spmv_row<VT, XT, SPMV_SET, false, RB><<<g1, 256, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    case SPMV_RESID: airg::note_launch(), k_spmv_row<VT, XT, SPMV_RESID, false, RB><<<g1, 256, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    case SPMV_ADD: airg::note_launch(), k_spmv_row<VT, XT, SPMV_ADD, false, RB><<<g1, 256, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    case SPMV_AXPB: airg::note_launch(), k_spmv_row<VT, XT, SPMV_AXPB, false, RB><<<g1, 256, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    default: airg::note_launch(), k_spmv_row<VT, XT, SPMV_ADDB, false, RB><<<g1, 256, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
  }
}

template <typename VT, typename XT, int LPR>
static void launch_spmv(int nrows, const int* rp, const int* ci, const VT* v, const XT* x, const XT* b, XT* y, int mode,
                        const int* w, XT* xf, cudaStream_t s, int rb, const XT* coef, bool keep) {
  if constexpr (LPR == 1) {
    if (rb == 8) launch_spmv_row<VT, XT, 8>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, coef, keep);
    else launch_spmv_row<VT, XT, 4>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, coef, keep);
    return;
  }
  const int grid = ceil_div(nrows, kSpmvThreads / LPR);
  if (w) {
    airg::note_launch(), k_spmv_vec<VT, XT, LPR, SPMV_RESID, true><<<grid, kSpmvThreads, 0, s>>>(nrows, rp, ci, v, x, b, y, w, xf, nullptr, keep);
    return;
  }
  switch (mode) {
    case SPMV_SET: airg::note_launch(), k_spmv_vec<VT, XT, LPR, SPMV_SET, false><<<grid, kSpmvThreads, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    case SPMV_RESID: airg::note_launch(), k_spmv_vec<VT, XT, LPR, SPMV_RESID, false><<<grid, kSpmvThreads, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    case SPMV_ADD: airg::note_launch(), k_spmv_vec<VT, XT, LPR, SPMV_ADD, false><<<grid, kSpmvThreads, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    case SPMV_AXPB: airg::note_launch(), k_spmv_vec<VT, XT, LPR, SPMV_AXPB, false><<<grid, kSpmvThreads, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
    default: airg::note_launch(), k_spmv_vec<VT, XT, LPR, SPMV_ADDB, false><<<grid, kSpmvThreads, 0, s>>>(nrows, rp, ci, v, x, b, y, nullptr, nullptr, coef, keep); break;
  }
}

template <typename VT, typename XT>
static void spmv_dispatch(int nrows, const int* rp, const int* ci, const VT* v, const XT* x, const XT* b, XT* y, int mode,
                          int lanes, const int* w, XT* xf, cudaStream_t s, int rb, const XT* coef, bool keep) {
  switch (lanes) {
    case 1: launch_spmv<VT, XT, 1>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, rb, coef, keep); break;
    case 2: launch_spmv<VT, XT, 2>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, rb, coef, keep); break;
    case 4: launch_spmv<VT, XT, 4>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, rb, coef, keep); break;
    case 8: launch_spmv<VT, XT, 8>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, rb, coef, keep); break;
    case 16: launch_spmv<VT, XT, 16>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, rb, coef, keep); break;
    default: launch_spmv<VT, XT, 32>(nrows, rp, ci, v, x, b, y, mode, w, xf, s, rb, coef, keep); break;
  }
}

double l2_keep_bytes() {
  static const double kb = [] {
    const char* e = getenv("AIRG_L2_KEEP_MB");
    return (e ? atof(e) : (double)kL2KeepMB) * 1048576.0;
  }();
  return kb;
}
template <typename VT>
static bool keep_in_l2(const DCsr& A) {
  return (double)A.nnz * (4.0 + sizeof(VT)) + 4.0 * (A.nrows + 1.0) <= l2_keep_bytes();
}

// Entries loaded per batch by the row-per-thread SpMV: 8 unless the rows average about 4 or fewer.
static int row_batch(const DCsr& A) { return (double)A.nnz > 4.5 * (double)A.nrows ? 8 : 4; }

// y = coef[0] b + A x (coef on the device): one Horner step of a matrix-free polynomial.
int dev_spmv_axpb(const DCsr& A, const double* x, const double* b, const double* coef, double* y, int lanes,
                  cudaStream_t s) {
  if (A.nrows <= 0) return AIRG_OK;
  if (A.sell) return sell_spmv(*A.sell, x, b, y, SPMV_AXPB, nullptr, nullptr, coef, s);
  spmv_dispatch<double, double>(A.nrows, A.rp, A.ci, A.v, x, b, y, SPMV_AXPB, lanes, nullptr, nullptr, s, row_batch(A),
                                coef, keep_in_l2<double>(A));
  KERNEL_CHECK();
  return AIRG_OK;
}

int dev_spmv(const DCsr& A, const double* x, const double* b, double* y, int mode, int lanes, cudaStream_t s) {
  if (A.nrows <= 0) return AIRG_OK;
  if (A.sell) return sell_spmv(*A.sell, x, b, y, mode, nullptr, nullptr, nullptr, s);
  spmv_dispatch<double, double>(A.nrows, A.rp, A.ci, A.v, x, b, y, mode, lanes, nullptr, nullptr, s, row_batch(A),
                                nullptr, keep_in_l2<double>(A));
  KERNEL_CHECK();
  return AIRG_OK;
}

// r = b_F - AF x with x_F replaced by the one-point prolongation of x_C; x_F is written too.
int dev_spmv_resid_prolong(const DCsr& AF, double* x, const int* w, const double* b, double* y, int lanes,
                           cudaStream_t s) {
  if (AF.nrows <= 0) return AIRG_OK;
  if (AF.sell) return sell_spmv(*AF.sell, x, b, y, SPMV_RESID, w, x, nullptr, s);
  spmv_dispatch<double, double>(AF.nrows, AF.rp, AF.ci, AF.v, x, b, y, SPMV_RESID, lanes, w, x, s, row_batch(AF),
                                nullptr, keep_in_l2<double>(AF));
  KERNEL_CHECK();
  return AIRG_OK;
}

// Mixed-precision V-cycle SpMVs: values stored as float (vt = 1) or bf16 (vt = 2), vectors and
// accumulation in float.
int dev_spmv_lo(const DCsr& A, const void* vals, int vt, const float* x, const float* b, float* y, int mode, int lanes,
                const int* w, cudaStream_t s) {
  if (A.nrows <= 0) return AIRG_OK;
  float* xf = w ? const_cast<float*>(x) : nullptr;
  if (A.sell && A.sell->v_lo && A.sell->vt == vt) return sell_spmv_lo(*A.sell, x, b, y, mode, w, xf, s);
  if (vt == 2)
    spmv_dispatch<__nv_bfloat16, float>(A.nrows, A.rp, A.ci, (const __nv_bfloat16*)vals, x, b, y, mode, lanes, w, xf, s,
                                        row_batch(A), nullptr, keep_in_l2<__nv_bfloat16>(A));
  else
    spmv_dispatch<float, float>(A.nrows, A.rp, A.ci, (const float*)vals, x, b, y, mode, lanes, w, xf, s, row_batch(A),
                                nullptr, keep_in_l2<float>(A));
  KERNEL_CHECK();
  return AIRG_OK;
}

__global__ void k_cast_d2f(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
__global__ void k_cast_d2bf(const double* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn((float)in[i]);
}
__global__ void k_cast_f2d(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
void dev_cast_d2f(const double* in, float* out, long long n, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_cast_d2f<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
}
void dev_cast_d2bf(const double* in, void* out, long long n, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_cast_d2bf<<<grid_for(n, 256), 256, 0, s>>>(in, (__nv_bfloat16*)out, n);
}
void dev_cast_f2d(const float* in, double* out, long long n, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_cast_f2d<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
}

__global__ void k_gather_prolong_f(float* x, int nf, const int* __restrict__ w) {
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    int c = w[f];
    x[f] = c >= 0 ? x[nf + c] : 0.0f;
  }
}
void dev_gather_prolong_f(float* x, int nf, const int* w, cudaStream_t s) {
  if (nf > 0) airg::note_launch(), k_gather_prolong_f<<<grid_for(nf, 256), 256, 0, s>>>(x, nf, w);
}

// Lanes per row for the SpMV: one thread per row (k_spmv_row) up to 12 entries per row on average,
// then LPR lanes per row (k_spmv_vec), about 6 entries per lane.
int pick_lanes(double L) {
  if (L <= 12.0) return 1;
  if (L <= 24.0) return 2;
  if (L <= 48.0) return 4;
  if (L <= 96.0) return 8;
  if (L <= 192.0) return 16;
  return 32;
}

// ------------------------------------------------------------------------------------------
// Small vector kernels
// ------------------------------------------------------------------------------------------
// y = x * (1/a): one multiply per element (an FP64 division per element would make this kernel
// bound by sm_103a's FP64 rate instead of by bandwidth)
__global__ void k_scale(const double* __restrict__ x, double inv, double* __restrict__ y, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}
void dev_scale(const double* x, double a, double* y, int n, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_scale<<<grid_for(n, 256), 256, 0, s>>>(x, 1.0 / a, y, n);
}

__global__ void k_permute(const double* __restrict__ in, const int* __restrict__ pos, double* __restrict__ out, int n,
                          bool inverse) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (inverse) out[i] = in[pos[i]];
    else out[pos[i]] = in[i];
  }
}
void dev_permute(const double* in, const int* pos, double* out, int n, bool inverse, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_permute<<<grid_for(n, 256), 256, 0, s>>>(in, pos, out, n, inverse);
}

__global__ void k_gather_prolong(double* x, int nf, const int* __restrict__ w) {
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    int c = w[f];
    x[f] = c >= 0 ? x[nf + c] : 0.0;
  }
}
void dev_gather_prolong(double* x, int nf, const int* w, cudaStream_t s) {
  if (nf > 0) airg::note_launch(), k_gather_prolong<<<grid_for(nf, 256), 256, 0, s>>>(x, nf, w);
}

// y = coef[0] r (add = false) or y += coef[0] r (add = true), coef on the device
__global__ void k_coef_axpy(const double* __restrict__ coef, const double* __restrict__ r, double* __restrict__ y, int n,
                            bool add) {
  const double a = coef[0];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = add ? y[i] + a * r[i] : a * r[i];
}
void dev_coef_axpy(const double* coef, const double* r, double* y, int n, bool add, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_coef_axpy<<<grid_for(n, 256), 256, 0, s>>>(coef, r, y, n, add);
}

// x += y
__global__ void k_add(const double* __restrict__ y, double* __restrict__ x, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += y[i];
}
void dev_add(const double* y, double* x, int n, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_add<<<grid_for(n, 256), 256, 0, s>>>(y, x, n);
}

__global__ void k_fill(double* x, double v, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}
void dev_fill(double* x, double v, int n, cudaStream_t s) {
  if (n > 0) airg::note_launch(), k_fill<<<grid_for(n, 256), 256, 0, s>>>(x, v, n);
}

}  // namespace airg
