// Sliced ELL (SELL-32-sigma) copies of the solve-phase operators and their SpMV.
//
// The solve's operators on the large levels have short rows (the 2D P1 DG top level holds rows of
// 3, 5 and 7 entries).  In CSR with one thread per row, the 32 lanes of a warp read 32 different
// rows, so every load instruction of columns and values touches many cache lines and the kernel is
// limited by L1 wavefronts and load latency rather than by DRAM.  Here the 32 rows of a warp are
// stored column-major (entry k of the 32 rows side by side), so each load instruction reads one
// contiguous 128-byte (columns) or 256-byte (values) segment.  Rows are sorted by length inside
// windows of kSellWindow rows before slicing, which keeps the padding to the slice's longest row
// near zero (about 1 % on the DG operators).  Each row's entries keep their CSR order and are
// accumulated with one FMA each from zero, in that order: the result is bitwise the CSR row
// kernel's.
#include <cuda_bf16.h>

#include <algorithm>

#include "airg_common.cuh"

namespace airg {

namespace {

constexpr int kSellBuckets = 64;  // row lengths >= 63 share the last bucket (unsorted among themselves)

// R entries of a slice from k0 on: loads first (R in flight per lane), then the gathers of x, then
// R FMAs in entry order.  R is a compile-time count so that exactly the slice's width in FP64
// FMAs is issued: on sm_103a the FP64 pipe takes about 64 cycles per warp instruction, so FMAs
// issued for entries past the width (predicated off) would cost as much as real ones.
// One FMA of a stored value (double, float or bf16) with the vector type XT (double or float).
__device__ __forceinline__ double sfma(double a, double x, double acc) { return fma(a, x, acc); }
__device__ __forceinline__ float sfma(float a, float x, float acc) { return fmaf(a, x, acc); }
__device__ __forceinline__ float sfma(__nv_bfloat16 a, float x, float acc) { return fmaf(__bfloat162float(a), x, acc); }

template <int R, bool PROLONG, typename VT, typename XT>
__device__ __forceinline__ XT sell_batch(const int* cs, const VT* vs, int k0, const XT* x, int nrows,
                                         const int* __restrict__ w, XT s, uint64_t pol) {
  int c[R];
  VT a[R];
  XT xv[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    c[t] = ld_pol(cs + (k0 + t) * 32, pol);
    a[t] = ld_pol(vs + (k0 + t) * 32, pol);
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
    if (c[t] >= 0) s = sfma(a[t], xv[t], s);
  return s;
}

// ------------------------------------------------------------------------------------------
// SpMV: one warp per slice (one launch wave after another; a persistent-warp variant that
// prefetched the next slice's offsets measured 40 % slower), lane l of slice s computes row
// perm[32 s + l].
// ------------------------------------------------------------------------------------------
// Eight resident CTAs per SM (32 registers) with 8-entry batches; the fused-prolongation variant,
// whose gathers hold more registers, takes 4-entry batches at six CTAs (40 registers).
template <int MODE, bool PROLONG, typename VT = double, typename XT = double>
__global__ void __launch_bounds__(256, PROLONG ? 6 : 8) k_spmv_sell(int nslices, int nrows, const int* __restrict__ sp,
                                                   const int* __restrict__ ci, const VT* __restrict__ v,
                                                   const int* __restrict__ perm, const XT* x, const XT* b,
                                                   XT* y, const int* __restrict__ w, XT* xf,
                                                   const XT* __restrict__ coef, bool keep) {
  const uint64_t pol = l2_policy(keep);
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nwarps) {
    const int beg = sp[sl];
    const int width = (sp[sl + 1] - beg) >> 5;  // warp-uniform
    const int row = perm[sl * 32 + lane];
    const int* cs = ci + beg + lane;
    const VT* vs = v + beg + lane;
    XT s = XT(0);
    int k0 = 0;
    if constexpr (PROLONG) {
      for (; k0 + 4 <= width; k0 += 4) s = sell_batch<4, PROLONG>(cs, vs, k0, x, nrows, w, s, pol);
      switch (width - k0) {  // warp-uniform remainder
        case 1: s = sell_batch<1, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 2: s = sell_batch<2, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 3: s = sell_batch<3, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        default: break;
      }
    } else {
      for (; k0 + 8 <= width; k0 += 8) s = sell_batch<8, PROLONG>(cs, vs, k0, x, nrows, w, s, pol);
      switch (width - k0) {  // warp-uniform remainder
        case 1: s = sell_batch<1, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 2: s = sell_batch<2, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 3: s = sell_batch<3, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 4: s = sell_batch<4, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 5: s = sell_batch<5, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 6: s = sell_batch<6, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        case 7: s = sell_batch<7, PROLONG>(cs, vs, k0, x, nrows, w, s, pol); break;
        default: break;
      }
    }
    if (row >= 0) {
      XT out;
      if (MODE == SPMV_SET) out = s;
      else if (MODE == SPMV_RESID) out = b[row] - s;
      else if (MODE == SPMV_ADD) out = y[row] + s;
      else if (MODE == SPMV_AXPB) out = coef[0] * b[row] + s;
      else out = b[row] + s;
      y[row] = out;
      if (PROLONG) {
        const int src = w[row];
        xf[row] = src >= 0 ? x[nrows + src] : XT(0);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Conversion
// ------------------------------------------------------------------------------------------
// One block of kSellWindow threads per window: a stable counting sort of the window's rows by
// descending length bucket.  Lanes of a warp that share a bucket are ranked with a match mask;
// per-warp bucket counts in shared memory give each warp's offset within a bucket.  Positions past
// the last row get perm -1 (bucket kSellBuckets, sorted last).
__global__ void __launch_bounds__(kSellWindow) k_sell_sort(int n, const int* __restrict__ rp, int* __restrict__ perm) {
  constexpr int NW = kSellWindow / 32, NB = kSellBuckets + 1;
  __shared__ int cnt[NW][NB];
  __shared__ int base[NB];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  for (int i = t; i < NW * NB; i += blockDim.x) cnt[i / NB][i % NB] = 0;
  __syncthreads();
  const long long row = (long long)blockIdx.x * kSellWindow + t;
  int key = kSellBuckets;
  if (row < n) {
    const int len = rp[row + 1] - rp[row];
    key = (kSellBuckets - 1) - min(len, kSellBuckets - 1);  // longer rows first
  }
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  if (rank == 0) cnt[wp][key] = __popc(peers);
  __syncthreads();
  if (t < NB) {  // exclusive scan over warps, per bucket
    int acc = 0;
    for (int q = 0; q < NW; ++q) {
      const int c = cnt[q][t];
      cnt[q][t] = acc;
      acc += c;
    }
    base[t] = acc;  // bucket total for now
  }
  __syncthreads();
  if (t == 0) {  // exclusive scan over buckets
    int acc = 0;
    for (int q = 0; q < NB; ++q) {
      const int c = base[q];
      base[q] = acc;
      acc += c;
    }
  }
  __syncthreads();
  const int pos = base[key] + cnt[wp][key] + rank;
  perm[(long long)blockIdx.x * kSellWindow + pos] = row < n ? (int)row : -1;
}

// Entries per slice (32 x its longest row).
__global__ void k_sell_width(int nslices, const int* __restrict__ rp, const int* __restrict__ perm, int* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nwarps) {
    const int row = perm[sl * 32 + lane];
    int len = row >= 0 ? rp[row + 1] - rp[row] : 0;
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) cnt[sl] = 32 * len;
  }
}

__global__ void k_sell_fill(int nslices, const int* __restrict__ rp, const int* __restrict__ aci,
                            const double* __restrict__ av, const int* __restrict__ perm, const int* __restrict__ sp,
                            int* __restrict__ ci, double* __restrict__ v) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < nslices; sl += nwarps) {
    const int beg = sp[sl], width = (sp[sl + 1] - beg) >> 5;
    const int row = perm[sl * 32 + lane];
    const int rb = row >= 0 ? rp[row] : 0, len = row >= 0 ? rp[row + 1] - rb : 0;
    for (int k = 0; k < width; ++k) {
      const bool in = k < len;
      ci[beg + k * 32 + lane] = in ? aci[rb + k] : -1;
      v[beg + k * 32 + lane] = in ? av[rb + k] : 0.0;
    }
  }
}

template <int MODE, bool PROLONG, typename VT, typename XT>
void launch_sell(const DSell& S, const VT* vals, const XT* x, const XT* b, XT* y, const int* w, XT* xf,
                 const XT* coef, cudaStream_t s) {
  const int grid = ceil_div(S.nslices, 256 / 32);
  // the same size rule as the CSR SpMVs: the copy's padded arrays against the L2 keep size
  const bool keep = (double)S.nnz_pad * (4.0 + sizeof(VT)) + 4.0 * (S.nslices + 1.0) + 4.0 * 32.0 * S.nslices <=
                    l2_keep_bytes();
  airg::note_launch(), k_spmv_sell<MODE, PROLONG, VT, XT><<<grid, 256, 0, s>>>(S.nslices, S.nrows, S.sp, S.ci, vals,
                                                                               S.perm, x, b, y, w, xf, coef, keep);
}

template <typename VT, typename XT>
void sell_dispatch(const DSell& S, const VT* vals, const XT* x, const XT* b, XT* y, int mode, const int* w, XT* xf,
                   const XT* coef, cudaStream_t s) {
  if (w) {
    launch_sell<SPMV_RESID, true>(S, vals, x, b, y, w, xf, coef, s);
    return;
  }
  switch (mode) {
    case SPMV_SET: launch_sell<SPMV_SET, false>(S, vals, x, b, y, w, xf, coef, s); break;
    case SPMV_RESID: launch_sell<SPMV_RESID, false>(S, vals, x, b, y, w, xf, coef, s); break;
    case SPMV_ADD: launch_sell<SPMV_ADD, false>(S, vals, x, b, y, w, xf, coef, s); break;
    case SPMV_AXPB: launch_sell<SPMV_AXPB, false>(S, vals, x, b, y, w, xf, coef, s); break;
    default: launch_sell<SPMV_ADDB, false>(S, vals, x, b, y, w, xf, coef, s); break;
  }
}

}  // namespace

bool want_sell(const DCsr& A) {
  // large operators whose rows the one-thread-per-row kernel would take (short rows)
  return A.nrows >= kSellMinRows && pick_lanes(A.nrows > 0 ? (double)A.nnz / A.nrows : 1.0) == 1;
}

int build_sell(const DCsr& A, DSell& out, Arena& own, Arena& tmp, cudaStream_t s) {
  const int n = A.nrows;
  const int nwin = ceil_div(n, kSellWindow);
  const int nslices = nwin * (kSellWindow / 32);
  out.nrows = n;
  out.nslices = nslices;
  AIRG_TRY(own.alloc(&out.perm, (size_t)nwin * kSellWindow));
  AIRG_TRY(own.alloc(&out.sp, (size_t)nslices + 1));
  int* cnt;
  AIRG_TRY(tmp.alloc(&cnt, (size_t)nslices));
  if (nwin > 0) airg::note_launch(), k_sell_sort<<<nwin, kSellWindow, 0, s>>>(n, A.rp, out.perm);
  KERNEL_CHECK();
  airg::note_launch(), k_sell_width<<<grid_for((long long)nslices * 32, 256), 256, 0, s>>>(nslices, A.rp, out.perm, cnt);
  KERNEL_CHECK();
  long long total = 0;
  AIRG_TRY(scan_i32(cnt, out.sp, nslices, tmp, s, &total));  // synchronises: total sizes the arrays
  if (total > 0x7fffffffLL) return AIRG_ERR_UNSUPPORTED;
  out.nnz_pad = total;
  AIRG_TRY(own.alloc(&out.ci, (size_t)std::max(total, 1LL)));
  AIRG_TRY(own.alloc(&out.v, (size_t)std::max(total, 1LL)));
  airg::note_launch(), k_sell_fill<<<grid_for((long long)nslices * 32, 256), 256, 0, s>>>(nslices, A.rp, A.ci, A.v,
                                                                                          out.perm, out.sp, out.ci, out.v);
  KERNEL_CHECK();
  return AIRG_OK;
}

int sell_spmv(const DSell& S, const double* x, const double* b, double* y, int mode, const int* w, double* xf,
              const double* coef, cudaStream_t s) {
  if (S.nslices <= 0) return AIRG_OK;
  sell_dispatch<double, double>(S, S.v, x, b, y, mode, w, xf, coef, s);
  KERNEL_CHECK();
  return AIRG_OK;
}

__global__ void k_sell_cast(long long n, const double* __restrict__ in, float* __restrict__ outf,
                            __nv_bfloat16* __restrict__ outb) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (outf) outf[i] = (float)in[i];
    else outb[i] = __float2bfloat16_rn((float)in[i]);
  }
}

int sell_cast_values(DSell& S, int vt, Arena& own, cudaStream_t s) {
  const long long n = std::max(S.nnz_pad, 1LL);
  if (vt == 1) {
    float* p;
    AIRG_TRY(own.alloc(&p, (size_t)n));
    airg::note_launch(), k_sell_cast<<<grid_for(n, 256), 256, 0, s>>>(S.nnz_pad, S.v, p, nullptr);
    S.v_lo = p;
  } else {
    __nv_bfloat16* p;
    AIRG_TRY(own.alloc(&p, (size_t)n));
    airg::note_launch(), k_sell_cast<<<grid_for(n, 256), 256, 0, s>>>(S.nnz_pad, S.v, nullptr, p);
    S.v_lo = p;
  }
  S.vt = vt;
  KERNEL_CHECK();
  return AIRG_OK;
}

int sell_spmv_lo(const DSell& S, const float* x, const float* b, float* y, int mode, const int* w, float* xf,
                 cudaStream_t s) {
  if (S.nslices <= 0) return AIRG_OK;
  if (S.vt == 2) sell_dispatch<__nv_bfloat16, float>(S, (const __nv_bfloat16*)S.v_lo, x, b, y, mode, w, xf, nullptr, s);
  else sell_dispatch<float, float>(S, (const float*)S.v_lo, x, b, y, mode, w, xf, nullptr, s);
  KERNEL_CHECK();
  return AIRG_OK;
}

}  // namespace airg
