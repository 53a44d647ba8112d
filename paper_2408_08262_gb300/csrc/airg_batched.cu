// Batched form: many independent systems (each with its own AIRG hierarchy) solved together.
//
// All systems' vectors are concatenated (system s at offset base_s, in its own nested solve
// numbering).  For every hierarchy depth d the level-d operators of all systems are concatenated
// into one CSR per role, with columns relabelled to absolute positions and a row -> position map,
// so each V-cycle step is a single launch over every system that has that level; the batched
// V-cycle is captured once as a CUDA graph.  The outer FGMRES runs all systems in lockstep with
// segmented (per-system) deterministic reductions and per-system Hessenberg/Givens on the host; a
// system that has converged is frozen.
#include <cmath>
#include <vector>

#include "airg_hier.cuh"

namespace airg {

namespace {

constexpr int kSegRows = 8192;  // rows per block of the segmented vector kernels
constexpr int kMaxCols = 32;

struct Group {
  DCsr A;              // concatenated operator (columns absolute, or group-row based for Ainv)
  int* map = nullptr;  // row -> position in the concatenated vectors
  int lanes = 1;
};

// Concatenation of all parts of a group in one launch: part p's rows go to rows r0_p.. of the
// group, its entries to z0_p.., its columns shifted by col_off_p; map[r] = map_off_p + local row.
// The part of a row is found by a binary search over the parts' first rows (parts with rows only).
struct ConcatPart {
  const int* rp;
  const int* ci;
  const double* v;
  int r0, z0, col_off, map_off, nrows;
};
__global__ void k_concat_parts(const ConcatPart* __restrict__ parts, int nparts, int rows, int nnz_total,
                               int* __restrict__ orp, int* __restrict__ oci, double* __restrict__ ov,
                               int* __restrict__ map) {
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0) orp[rows] = nnz_total;
  for (long long rr = t0; rr < rows; rr += (long long)gridDim.x * blockDim.x) {
    const int r = (int)rr;
    int lo = 0, hi = nparts - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (parts[mid].r0 <= r) lo = mid;
      else hi = mid - 1;
    }
    const ConcatPart& P = parts[lo];
    const int i = r - P.r0;
    const int b = P.rp[i], e = P.rp[i + 1];
    orp[r] = P.z0 + b;
    for (int k = b; k < e; ++k) {
      oci[P.z0 + k] = P.ci[k] + P.col_off;
      ov[P.z0 + k] = P.v[k];
    }
    if (map) map[r] = P.map_off + i;
  }
}

// x[dst[i]] = src[i] >= 0 ? x[src[i]] : 0   (one-point prolongation over the batch)
__global__ void k_gather_pos(double* x, const int* __restrict__ dst, const int* __restrict__ src, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int sidx = src[i];
    x[dst[i]] = sidx >= 0 ? x[sidx] : 0.0;
  }
}
__global__ void k_prolong_src(int nf, const int* __restrict__ w, int dst0, int src0, int* __restrict__ dst,
                              int* __restrict__ src, int out0) {
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    dst[out0 + f] = dst0 + (int)f;
    const int c = w[f];
    src[out0 + f] = c >= 0 ? src0 + c : -1;
  }
}
// y[r] = x[map[r]]
__global__ void k_gather_map(const double* __restrict__ x, const int* __restrict__ map, double* __restrict__ y, int n) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    y[r] = x[map[r]];
}

// SpMV with a row map (same scheme as the single-system kernels: the LPR lanes of a row read its
// entries directly, 4 per batch, accumulate with FMAs and combine by a butterfly):
//   SET: y[map r] = s;  RESID: y[r] = b[map r] - s;  ADD: y[map r] += s;  ADDB: y[map r] = b[map r] + s
template <int LPR, int MODE>
__global__ void __launch_bounds__(256) k_spmv_mapped(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                                                     const double* __restrict__ v, const double* x, const double* b,
                                                     double* y, const int* __restrict__ map) {
  constexpr int GPW = 32 / LPR;
  const int lane = threadIdx.x % LPR, grp = (threadIdx.x & 31) / LPR;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * GPW; base < nrows; base += nwarps * GPW) {  // warp-uniform
    const long long rr = base + grp;
    const bool act = rr < nrows;
    const int row = act ? (int)rr : 0;
    const int rb = act ? rp[row] : 0, re = act ? rp[row + 1] : 0;
    double s = 0.0;
    for (int k0 = rb + lane; k0 < re; k0 += 4 * LPR) {
      int c[4];
      double a[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int k = k0 + t * LPR;
        c[t] = (k < re) ? __ldcs(ci + k) : -1;
        a[t] = (k < re) ? __ldcs(v + k) : 0.0;
      }
      double xv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) xv[t] = (c[t] >= 0) ? __ldg(x + c[t]) : 0.0;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (c[t] >= 0) s = fma(a[t], xv[t], s);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LPR);
    if (act && lane == 0) {
      const int m = map[row];
      if (MODE == SPMV_SET) y[m] = s;
      else if (MODE == SPMV_RESID) y[row] = b[m] - s;
      else if (MODE == SPMV_ADD) y[m] = y[m] + s;
      else y[m] = b[m] + s;
    }
  }
}

template <int LPR>
void launch_mapped(const Group& g, const double* x, const double* b, double* y, int mode, cudaStream_t s) {
  const int grid = ceil_div(g.A.nrows, 256 / LPR);
  switch (mode) {
    case SPMV_SET: airg::note_launch(), k_spmv_mapped<LPR, SPMV_SET><<<grid, 256, 0, s>>>(g.A.nrows, g.A.rp, g.A.ci, g.A.v, x, b, y, g.map); break;
    case SPMV_RESID: airg::note_launch(), k_spmv_mapped<LPR, SPMV_RESID><<<grid, 256, 0, s>>>(g.A.nrows, g.A.rp, g.A.ci, g.A.v, x, b, y, g.map); break;
    case SPMV_ADD: airg::note_launch(), k_spmv_mapped<LPR, SPMV_ADD><<<grid, 256, 0, s>>>(g.A.nrows, g.A.rp, g.A.ci, g.A.v, x, b, y, g.map); break;
    default: airg::note_launch(), k_spmv_mapped<LPR, SPMV_ADDB><<<grid, 256, 0, s>>>(g.A.nrows, g.A.rp, g.A.ci, g.A.v, x, b, y, g.map); break;
  }
}
int spmv_mapped(const Group& g, const double* x, const double* b, double* y, int mode, cudaStream_t s) {
  if (g.A.nrows <= 0) return AIRG_OK;
  switch (g.lanes) {
    case 1: launch_mapped<1>(g, x, b, y, mode, s); break;
    case 2: launch_mapped<2>(g, x, b, y, mode, s); break;
    case 4: launch_mapped<4>(g, x, b, y, mode, s); break;
    case 8: launch_mapped<8>(g, x, b, y, mode, s); break;
    case 16: launch_mapped<16>(g, x, b, y, mode, s); break;
    default: launch_mapped<32>(g, x, b, y, mode, s); break;
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

// ---- segmented (per-system) vector kernels; block b covers rows [lo_b, hi_b) of system sys_b ----
struct SegTab {
  int nblk = 0;
  int *sys = nullptr, *sys_first = nullptr, *sys_last = nullptr;  // per block / per system block range
  long long *lo = nullptr, *hi = nullptr;
  double* partial = nullptr;  // [nblk][kMaxCols + 2]
  unsigned* counter = nullptr;  // [nsys]
};

// w -= V hsub[sys] (if hsub); dots[sys][k] = V_k . w (k < ncols, if dots); nrm[sys] = w . w (if nrm)
template <int NC>
__global__ void __launch_bounds__(256) k_seg_gs(const double* __restrict__ V, long long ldv, int ncols, double* w,
                                                SegTab t, const double* __restrict__ hsub, double* dots, double* nrm) {
  constexpr int NV = NC + 1;
  __shared__ double sh[NC];
  __shared__ double red[8][NV];
  __shared__ bool last;
  const int b = blockIdx.x, sys = t.sys[b];
  const int nd = dots ? ncols : 0;
  if (hsub)
    for (int k = threadIdx.x; k < ncols; k += blockDim.x) sh[k] = hsub[sys * (kMaxCols + 2) + k];
  __syncthreads();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  // NC == ncols (one instance per column count): no FP64 instruction is issued for an absent
  // column -- sm_103a's FP64 pipe spends a warp instruction's time on predicated-off lanes too
  const bool want = nd > 0;
  for (long long r = t.lo[b] + threadIdx.x; r < t.hi[b]; r += blockDim.x) {
    double wr = w[r];
    if (hsub) {
      double sub = 0.0;
#pragma unroll
      for (int k = 0; k < NC; ++k) sub += V[(size_t)k * ldv + r] * sh[k];
      wr -= sub;
      w[r] = wr;
    }
    if (want) {
#pragma unroll
      for (int k = 0; k < NC; ++k) acc[k] += V[(size_t)k * ldv + r] * wr;
    }
    acc[NC] += wr * wr;
  }
#pragma unroll
  for (int k = 0; k < NC; ++k)
    if (k == nd) acc[k] = acc[NC];
  const int nv = nd + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
    if (k < nv) {
      double v = acc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][k] = v;
    }
  __syncthreads();
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < nw; ++q) v += red[q][k];
    t.partial[(size_t)b * (kMaxCols + 2) + k] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nb = (unsigned)(t.sys_last[sys] - t.sys_first[sys] + 1);
    last = (atomicAdd(t.counter + sys, 1u) == nb - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double v = 0.0;
    for (int q = t.sys_first[sys]; q <= t.sys_last[sys]; ++q) v += ((volatile double*)t.partial)[(size_t)q * (kMaxCols + 2) + k];
    if (k < nd) dots[sys * (kMaxCols + 2) + k] = v;
    else if (nrm) nrm[sys] = v;
  }
  if (threadIdx.x == 0) t.counter[sys] = 0u;
}

// y = x * f[sys]
__global__ void k_seg_scale(const double* __restrict__ x, double* __restrict__ y, SegTab t, const double* __restrict__ f) {
  const int b = blockIdx.x;
  const double a = f[t.sys[b]];
  for (long long r = t.lo[b] + threadIdx.x; r < t.hi[b]; r += blockDim.x) y[r] = x[r] * a;
}
// x += sum_k V_k y[sys][k] for k < cnt[sys]
__global__ void k_seg_axpy(const double* __restrict__ V, long long ldv, double* __restrict__ x, SegTab t,
                           const double* __restrict__ y, const int* __restrict__ cnt) {
  const int b = blockIdx.x, sys = t.sys[b];
  const int c = cnt[sys];
  for (long long r = t.lo[b] + threadIdx.x; r < t.hi[b]; r += blockDim.x) {
    double a = x[r];
    for (int k = 0; k < c; ++k) a += y[sys * (kMaxCols + 2) + k] * V[(size_t)k * ldv + r];
    x[r] = a;
  }
}
// out[base + pos[i]] = in_s[i] (forward) or out_s[i] = in[base + pos[i]] (inverse)
__global__ void k_perm_in(const double* __restrict__ in, const int* __restrict__ pos, double* __restrict__ out,
                          long long base, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[base + (pos ? pos[i] : i)] = in[i];
}
__global__ void k_perm_out(const double* __restrict__ in, const int* __restrict__ pos, double* __restrict__ out,
                           long long base, int n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = in[base + (pos ? pos[i] : i)];
}

}  // namespace
}  // namespace airg

using namespace airg;

struct airg_batch {
  int nsys = 0;
  std::deque<std::vector<airg::ConcatPart>> part_tables;  // host tables of the concatenation launches
  cudaStream_t s = nullptr;
  Arena mem;
  std::vector<airg_hierarchy*> H;
  std::vector<long long> base;
  long long N = 0;
  int D = 0;  // deepest level index + 1
  std::vector<Group> Z, AF, Ai, CA, CAi;  // per depth
  std::vector<int*> pdst, psrc;
  std::vector<int> pn;
  Group A0;
  SegTab seg;
  int restart_alloc = 0;
  double *V = nullptr, *Zk = nullptr, *w = nullptr, *r = nullptr, *bwork = nullptr, *rtmp = nullptr, *bp = nullptr,
         *xp = nullptr, *gin = nullptr, *gout = nullptr, *dsc = nullptr, *hsc = nullptr;
  int* dcnt = nullptr;
  cudaGraphExec_t vg = nullptr;
  cudaStream_t cap = nullptr;
  long long vg_kernels = 0;
  // SpMV autotuner: lanes per row of every grouped operator picked by timing (AIRG_NO_AUTOTUNE=1:
  // the row-length rule alone); scratch vectors for the trial launches
  bool tune = true;
  double *tx = nullptr, *ty = nullptr;
  std::vector<std::pair<int, int>> tuned;  // (rule's lanes, chosen lanes) per tuned group
};

namespace {

// The autotuner: the row-length rule's lanes per row and its two neighbours (half and twice as
// many lanes) run on the group's operator (SET into scratch vectors, one untimed launch then
// kTuneReps timed with CUDA events on the batch's stream), and the fastest is kept.  Three
// candidates rather than all six keep the creation of a batch cheap next to its solves.  Groups below kTuneMinRows rows keep the
// row-length rule: their launches are latency-bound whatever the variant.  The row sums of
// different variants round differently, so a batch's results can change in the last bits with the
// variants chosen.
constexpr long long kTuneMinRows = 16384;
constexpr int kTuneReps = 2;

int tune_lanes(airg_batch* B, Group& g) {
  cudaStream_t s = B->s;
  if (!B->tx) {
    AIRG_TRY(B->mem.alloc(&B->tx, (size_t)std::max(B->N, 1LL)));
    AIRG_TRY(B->mem.alloc(&B->ty, (size_t)std::max(B->N, 1LL)));
    CU_TRY(cudaMemsetAsync(B->tx, 0, sizeof(double) * (size_t)std::max(B->N, 1LL), s));
  }
  cudaEvent_t e0, e1;
  CU_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AIRG_ERR_CUDA;
  }
  const int rule = g.lanes;
  int best = rule;
  float best_ms = 0.f;
  int rc = AIRG_OK;
  // the row-length rule's choice and its two neighbours (half and twice the lanes per row)
  const int cand[3] = {rule, rule / 2, rule * 2};
  for (int c = 0; c < 3 && rc == AIRG_OK; ++c) {
    const int lanes = cand[c];
    if (lanes < 1 || lanes > 32) continue;
    g.lanes = lanes;
    rc = spmv_mapped(g, B->tx, nullptr, B->ty, SPMV_SET, s);
    if (rc == AIRG_OK) rc = cuda_status(cudaEventRecord(e0, s));
    for (int r = 0; r < kTuneReps && rc == AIRG_OK; ++r) rc = spmv_mapped(g, B->tx, nullptr, B->ty, SPMV_SET, s);
    if (rc == AIRG_OK) rc = cuda_status(cudaEventRecord(e1, s));
    if (rc == AIRG_OK) rc = cuda_status(cudaEventSynchronize(e1));
    float ms = 0.f;
    if (rc == AIRG_OK) rc = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
    if (rc == AIRG_OK && (c == 0 || ms < best_ms)) {
      best_ms = ms;
      best = lanes;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.lanes = best;
  B->tuned.push_back({rule, best});
  return rc;
}

int concat_group(airg_batch* B, std::vector<std::pair<int, const DCsr*>>& parts, std::vector<int>& col_off,
                 std::vector<int>& map_off, Group& g) {
  cudaStream_t s = B->s;
  long long rows = 0, nnz = 0;
  for (auto& p : parts) {
    rows += p.second->nrows;
    nnz += p.second->nnz;
  }
  if (rows == 0) return AIRG_OK;
  if (rows > 0x7fffffffLL || nnz > 0x7fffffffLL) return AIRG_ERR_UNSUPPORTED;
  AIRG_TRY(B->mem.csr(g.A, (int)rows, (int)B->N, (int)nnz));
  AIRG_TRY(B->mem.alloc(&g.map, (size_t)rows));
  // one launch per group; the part table stays alive on the host until the build synchronises
  B->part_tables.emplace_back();
  std::vector<ConcatPart>& tab = B->part_tables.back();
  long long r0 = 0, z0 = 0;
  for (size_t q = 0; q < parts.size(); ++q) {
    const DCsr& M = *parts[q].second;
    if (M.nrows > 0) tab.push_back({M.rp, M.ci, M.v, (int)r0, (int)z0, col_off[q], map_off[q], M.nrows});
    r0 += M.nrows;
    z0 += M.nnz;
  }
  ConcatPart* dtab;
  AIRG_TRY(B->mem.alloc(&dtab, tab.size()));
  CU_TRY(cudaMemcpyAsync(dtab, tab.data(), sizeof(ConcatPart) * tab.size(), cudaMemcpyHostToDevice, s));
  airg::note_launch(), k_concat_parts<<<grid_for(rows, 256), 256, 0, s>>>(dtab, (int)tab.size(), (int)rows, (int)nnz,
                                                                           g.A.rp, g.A.ci, g.A.v, g.map);
  g.lanes = pick_lanes((double)nnz / (double)rows);
  KERNEL_CHECK();
  if (B->tune && rows >= kTuneMinRows) AIRG_TRY(tune_lanes(B, g));
  return AIRG_OK;
}

int batch_build(airg_batch* B) {
  cudaStream_t s = B->s;
  const int ns = B->nsys;
  B->base.resize(ns);
  long long N = 0;
  int D = 0;
  for (int q = 0; q < ns; ++q) {
    B->base[q] = N;
    N += B->H[q]->n0;
    D = std::max(D, (int)B->H[q]->lv.size());
  }
  if (N > 0x7fffffffLL) return AIRG_ERR_UNSUPPORTED;
  B->N = N;
  B->D = D;
  B->Z.resize(D);
  B->AF.resize(D);
  B->Ai.resize(D);
  B->CA.resize(D);
  B->CAi.resize(D);
  B->pdst.assign(D, nullptr);
  B->psrc.assign(D, nullptr);
  B->pn.assign(D, 0);
  for (int d = 0; d < D; ++d) {
    std::vector<std::pair<int, const DCsr*>> pz, paf, pai, pca, pcai;
    std::vector<int> cz, mz, caf, maf, cai, mai, cca, mca, ccai, mcai;
    int rows_f = 0, rows_c = 0, npro = 0;
    for (int q = 0; q < ns; ++q) {
      airg_hierarchy* H = B->H[q];
      if (d >= (int)H->lv.size()) continue;
      const SolveLevel& S = H->lv[d];
      const int o = (int)(B->base[q] + S.off);
      if (S.coarsest) {
        pca.push_back({q, &S.A});
        cca.push_back(o);
        mca.push_back(o);
        pcai.push_back({q, &S.Ainv});
        ccai.push_back(rows_c);  // Ainv_L columns index the group's work vector
        mcai.push_back(o);
        rows_c += S.n;
      } else {
        pz.push_back({q, &S.Z});
        cz.push_back(o);  // Z columns: the level's F entries of b
        mz.push_back(o + S.nf);  // rows: the level's C part = next level's vector
        paf.push_back({q, &S.AF});
        caf.push_back(o);
        maf.push_back(o);
        pai.push_back({q, &S.Ainv});
        cai.push_back(rows_f);  // Ainv columns index the group's residual vector
        mai.push_back(o);
        rows_f += S.nf;
        npro += S.nf;
      }
    }
    AIRG_TRY(concat_group(B, pz, cz, mz, B->Z[d]));
    AIRG_TRY(concat_group(B, paf, caf, maf, B->AF[d]));
    AIRG_TRY(concat_group(B, pai, cai, mai, B->Ai[d]));
    AIRG_TRY(concat_group(B, pca, cca, mca, B->CA[d]));
    AIRG_TRY(concat_group(B, pcai, ccai, mcai, B->CAi[d]));
    if (npro > 0) {
      AIRG_TRY(B->mem.alloc(&B->pdst[d], npro));
      AIRG_TRY(B->mem.alloc(&B->psrc[d], npro));
      int o0 = 0;
      for (int q = 0; q < ns; ++q) {
        airg_hierarchy* H = B->H[q];
        if (d >= (int)H->lv.size() || H->lv[d].coarsest) continue;
        const SolveLevel& S = H->lv[d];
        const int o = (int)(B->base[q] + S.off);
        if (S.nf > 0)
          airg::note_launch(), k_prolong_src<<<grid_for(S.nf, 256), 256, 0, s>>>(S.nf, S.w, o, o + S.nf, B->pdst[d], B->psrc[d], o0);
        o0 += S.nf;
      }
      B->pn[d] = npro;
    }
    KERNEL_CHECK();
  }
  // top-level operators, block diagonal
  {
    std::vector<std::pair<int, const DCsr*>> p0;
    std::vector<int> c0, m0;
    for (int q = 0; q < ns; ++q) {
      p0.push_back({q, &B->H[q]->A0s});
      c0.push_back((int)B->base[q]);
      m0.push_back((int)B->base[q]);
    }
    AIRG_TRY(concat_group(B, p0, c0, m0, B->A0));
  }
  // segment table
  std::vector<int> bsys, first(ns), lastb(ns);
  std::vector<long long> lo, hi;
  for (int q = 0; q < ns; ++q) {
    const long long n = B->H[q]->n0;
    first[q] = (int)bsys.size();
    for (long long r = 0; r < n || (r == 0 && n == 0); r += kSegRows) {
      bsys.push_back(q);
      lo.push_back(B->base[q] + r);
      hi.push_back(B->base[q] + std::min(n, r + kSegRows));
      if (n == 0) break;
    }
    lastb[q] = (int)bsys.size() - 1;
  }
  SegTab& t = B->seg;
  t.nblk = (int)bsys.size();
  AIRG_TRY(B->mem.alloc(&t.sys, t.nblk));
  AIRG_TRY(B->mem.alloc(&t.lo, t.nblk));
  AIRG_TRY(B->mem.alloc(&t.hi, t.nblk));
  AIRG_TRY(B->mem.alloc(&t.sys_first, ns));
  AIRG_TRY(B->mem.alloc(&t.sys_last, ns));
  AIRG_TRY(B->mem.alloc(&t.partial, (size_t)t.nblk * (kMaxCols + 2)));
  AIRG_TRY(B->mem.alloc(&t.counter, ns));
  CU_TRY(cudaMemcpyAsync(t.sys, bsys.data(), sizeof(int) * t.nblk, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemcpyAsync(t.lo, lo.data(), sizeof(long long) * t.nblk, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemcpyAsync(t.hi, hi.data(), sizeof(long long) * t.nblk, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemcpyAsync(t.sys_first, first.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemcpyAsync(t.sys_last, lastb.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
  CU_TRY(cudaMemsetAsync(t.counter, 0, sizeof(unsigned) * ns, s));
  CU_TRY(cudaStreamSynchronize(s));
  return AIRG_OK;
}

// Batched V-cycle in the concatenated nested layout: gin -> gout.
int batch_vcycle(airg_batch* B, const double* b0, double* x0) {
  cudaStream_t s = B->s;
  const int D = B->D;
  for (int d = 0; d < D; ++d)  // restriction: b_{d+1} = b_C + Z b_F for every system with a level d
    AIRG_TRY(spmv_mapped(B->Z[d], d == 0 ? b0 : B->bwork, d == 0 ? b0 : B->bwork, B->bwork, SPMV_ADDB, s));
  for (int d = D - 1; d >= 0; --d) {
    const double* bd = d == 0 ? b0 : B->bwork;
    const Group& CA = B->CA[d];
    const Group& CAi = B->CAi[d];
    if (CAi.A.nrows > 0) {  // systems whose coarsest level is d: x = Ainv b, then x += Ainv (b - A x)
      airg::note_launch(), k_gather_map<<<grid_for(CAi.A.nrows, 256), 256, 0, s>>>(bd, CAi.map, B->rtmp, CAi.A.nrows);
      AIRG_TRY(spmv_mapped(CAi, B->rtmp, nullptr, x0, SPMV_SET, s));
      for (int it = 1; it < B->H[0]->p.coarse_iters; ++it) {
        AIRG_TRY(spmv_mapped(CA, x0, bd, B->rtmp, SPMV_RESID, s));
        AIRG_TRY(spmv_mapped(CAi, B->rtmp, nullptr, x0, SPMV_ADD, s));
      }
    }
    if (B->AF[d].A.nrows > 0) {  // prolongation and up F-point smoothing
      airg::note_launch(), k_gather_pos<<<grid_for(B->pn[d], 256), 256, 0, s>>>(x0, B->pdst[d], B->psrc[d], B->pn[d]);
      for (int sm = 0; sm < B->H[0]->p.n_smooth_up; ++sm) {
        AIRG_TRY(spmv_mapped(B->AF[d], x0, bd, B->rtmp, SPMV_RESID, s));
        AIRG_TRY(spmv_mapped(B->Ai[d], B->rtmp, nullptr, x0, SPMV_ADD, s));
      }
    }
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

int batch_graph(airg_batch* B) {
  if (B->vg) return AIRG_OK;
  if (!B->cap) CU_TRY(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  cudaStream_t saved = B->s;
  B->s = B->cap;
  const long long l0 = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? batch_vcycle(B, B->gin, B->gout) : cuda_status(e);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(B->cap, &g) : cudaSuccess;
  B->vg_kernels = g_launches.load() - l0;
  g_launches.fetch_sub(B->vg_kernels);
  B->s = saved;
  if (rc == AIRG_OK && e2 != cudaSuccess) rc = cuda_status(e2);
  if (rc == AIRG_OK) rc = cuda_status(cudaGraphInstantiate(&B->vg, g, 0));
  if (g) cudaGraphDestroy(g);
  if (rc != AIRG_OK) {
    cudaGetLastError();
    B->vg = nullptr;
  }
  return rc;
}

int seg_gs(airg_batch* B, const double* V, int ncols, double* w, const double* hsub, double* dots, double* nrm) {
  const SegTab& t = B->seg;
  const long long ld = B->N;
  if (ncols == 0 && hsub) return AIRG_ERR_ARG;
  switch (ncols) {
    case 0:  // the norm alone (no columns to subtract or project on)
      airg::note_launch(), k_seg_gs<1><<<t.nblk, 256, 0, B->s>>>(V, ld, 0, w, t, nullptr, dots, nrm);
      break;
#define AIRG_SEG_GS(N) \
  case N: airg::note_launch(), k_seg_gs<N><<<t.nblk, 256, 0, B->s>>>(V, ld, ncols, w, t, hsub, dots, nrm); break;
    AIRG_SEG_GS(1) AIRG_SEG_GS(2) AIRG_SEG_GS(3) AIRG_SEG_GS(4) AIRG_SEG_GS(5) AIRG_SEG_GS(6) AIRG_SEG_GS(7)
    AIRG_SEG_GS(8) AIRG_SEG_GS(9) AIRG_SEG_GS(10) AIRG_SEG_GS(11) AIRG_SEG_GS(12) AIRG_SEG_GS(13) AIRG_SEG_GS(14)
    AIRG_SEG_GS(15) AIRG_SEG_GS(16) AIRG_SEG_GS(17) AIRG_SEG_GS(18) AIRG_SEG_GS(19) AIRG_SEG_GS(20) AIRG_SEG_GS(21)
    AIRG_SEG_GS(22) AIRG_SEG_GS(23) AIRG_SEG_GS(24) AIRG_SEG_GS(25) AIRG_SEG_GS(26) AIRG_SEG_GS(27) AIRG_SEG_GS(28)
    AIRG_SEG_GS(29) AIRG_SEG_GS(30) AIRG_SEG_GS(31) AIRG_SEG_GS(32)
#undef AIRG_SEG_GS
    default: return AIRG_ERR_ARG;
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

}  // namespace

extern "C" {

int airg_batch_create(airg_hierarchy* const* Hs, int nsys, airg_stream_t stream, airg_batch** out) {
  if (!out || !Hs || nsys <= 0) return AIRG_ERR_ARG;
  *out = nullptr;
  for (int q = 0; q < nsys; ++q) {
    if (!Hs[q] || Hs[q]->vt != 0) return AIRG_ERR_ARG;  // FP64 hierarchies
    if (Hs[q]->p.coarse_iters != Hs[0]->p.coarse_iters || Hs[q]->p.n_smooth_up != Hs[0]->p.n_smooth_up) return AIRG_ERR_ARG;
    // the batched V-cycle applies assembled inverses and one-point prolongators
    if (Hs[q]->p.matrix_free || Hs[q]->p.ideal_prolong) return AIRG_ERR_ARG;
  }
  airg_batch* B = new (std::nothrow) airg_batch;
  if (!B) return AIRG_ERR_OOM;
  {
    const char* t = getenv("AIRG_NO_AUTOTUNE");
    B->tune = !(t && t[0] == '1');
  }
  B->nsys = nsys;
  B->s = (cudaStream_t)stream;
  B->mem.s = B->s;
  B->H.assign(Hs, Hs + nsys);
  int rc = batch_build(B);
  if (rc != AIRG_OK) {
    airg_batch_free(B);
    return rc;
  }
  *out = B;
  return AIRG_OK;
}

void airg_batch_free(airg_batch* B) {
  if (!B) return;
  cudaStreamSynchronize(B->s);
  if (B->vg) cudaGraphExecDestroy(B->vg);
  if (B->cap) cudaStreamDestroy(B->cap);
  B->mem.release();
  cudaStreamSynchronize(B->s);
  if (B->hsc) cudaFreeHost(B->hsc);
  delete B;
}

int airg_batch_tuned(const airg_batch* B, int* rule_lanes, int* chosen_lanes, int cap) {
  if (!B || cap < 0) return AIRG_ERR_ARG;
  const int n = (int)B->tuned.size();
  for (int k = 0; k < n && k < cap; ++k) {
    if (rule_lanes) rule_lanes[k] = B->tuned[k].first;
    if (chosen_lanes) chosen_lanes[k] = B->tuned[k].second;
  }
  return n;
}

int airg_solve_batched(airg_batch* B, const double* const* b, double* const* x, const airg_solve_opts* o,
                       airg_solve_info* infos, airg_stream_t stream) {
  if (!B || !b || !x || !o || !infos) return AIRG_ERR_ARG;
  if (o->outer != AIRG_OUTER_FGMRES || o->restart < 1 || o->restart > kMaxCols - 2 || o->max_it < 0) return AIRG_ERR_ARG;
  B->s = (cudaStream_t)stream;
  B->mem.s = B->s;
  cudaStream_t s = B->s;
  const int ns = B->nsys, restart = o->restart;
  const long long N = B->N;
  if (B->restart_alloc < restart) {
    AIRG_TRY(B->mem.alloc(&B->V, (size_t)N * (restart + 1)));
    AIRG_TRY(B->mem.alloc(&B->Zk, (size_t)N * restart));
    B->restart_alloc = restart;
  }
  if (!B->w) {
    AIRG_TRY(B->mem.alloc(&B->w, N));
    AIRG_TRY(B->mem.alloc(&B->r, N));
    AIRG_TRY(B->mem.alloc(&B->bwork, N));
    AIRG_TRY(B->mem.alloc(&B->rtmp, N));
    AIRG_TRY(B->mem.alloc(&B->bp, N));
    AIRG_TRY(B->mem.alloc(&B->xp, N));
    AIRG_TRY(B->mem.alloc(&B->gin, N));
    AIRG_TRY(B->mem.alloc(&B->gout, N));
    AIRG_TRY(B->mem.alloc(&B->dsc, (size_t)ns * (kMaxCols + 2) * 4 + 2 * ns));
    AIRG_TRY(B->mem.alloc(&B->dcnt, ns));
    CU_TRY(cudaMallocHost((void**)&B->hsc, sizeof(double) * ((size_t)ns * (kMaxCols + 2) * 4 + 2 * ns)));
  }
  AIRG_TRY(batch_graph(B));
  const int CS = kMaxCols + 2;
  double* dH1 = B->dsc;
  double* dH2 = B->dsc + (size_t)ns * CS;
  double* dY = B->dsc + (size_t)ns * CS * 2;
  double* dF = B->dsc + (size_t)ns * CS * 3;  // per-system factors
  double* dN = dF + ns;                       // per-system norms
  double* hH1 = B->hsc;
  double* hH2 = B->hsc + (size_t)ns * CS;
  double* hN = B->hsc + (size_t)ns * CS * 3 + ns;
  auto read = [&]() -> int {
    CU_TRY(cudaMemcpyAsync(B->hsc, B->dsc, sizeof(double) * ((size_t)ns * CS * 4 + 2 * ns), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    return AIRG_OK;
  };
  // inputs into the concatenated solve numbering
  for (int q = 0; q < ns; ++q) {
    airg_hierarchy* H = B->H[q];
    if (H->n0 > 0) {
      airg::note_launch(), k_perm_in<<<grid_for(H->n0, 256), 256, 0, s>>>(b[q], H->pos0, B->bp, B->base[q], H->n0);
      if (o->x0_zero) CU_TRY(cudaMemsetAsync(B->xp + B->base[q], 0, sizeof(double) * H->n0, s));
      else airg::note_launch(), k_perm_in<<<grid_for(H->n0, 256), 256, 0, s>>>(x[q], H->pos0, B->xp, B->base[q], H->n0);
    }
  }
  KERNEL_CHECK();
  AIRG_TRY(seg_gs(B, B->bp, 0, B->bp, nullptr, nullptr, dN));
  AIRG_TRY(read());
  std::vector<double> bn(ns), beta(ns), relres(ns);
  std::vector<int> iters(ns, 0), status(ns, AIRG_OK), done(ns, 0);
  for (int q = 0; q < ns; ++q) bn[q] = std::sqrt(hN[q]);
  auto residual = [&]() -> int {
    AIRG_TRY(spmv_mapped(B->A0, B->xp, B->bp, B->r, SPMV_RESID, s));
    AIRG_TRY(seg_gs(B, B->r, 0, B->r, nullptr, nullptr, dN));
    AIRG_TRY(read());
    for (int q = 0; q < ns; ++q) {
      beta[q] = std::sqrt(hN[q]);
      relres[q] = bn[q] > 0 ? beta[q] / bn[q] : 0.0;
    }
    return AIRG_OK;
  };
  AIRG_TRY(residual());
  std::vector<double> Hh((size_t)ns * (restart + 1) * restart), cs((size_t)ns * restart), sn((size_t)ns * restart),
      g((size_t)ns * (restart + 1)), fac(ns), Y((size_t)ns * CS, 0.0);
  std::vector<int> k_s(ns), live(ns), cnt(ns);
  while (true) {
    int nlive = 0;
    for (int q = 0; q < ns; ++q) {
      live[q] = 0;
      if (done[q]) continue;
      if (!(relres[q] == relres[q]) || std::isinf(relres[q])) { status[q] = AIRG_ERR_NAN; done[q] = 1; continue; }
      if (relres[q] <= o->rtol || bn[q] == 0.0) { done[q] = 1; continue; }
      if (iters[q] >= o->max_it) { status[q] = AIRG_NOT_CONVERGED; done[q] = 1; continue; }
      live[q] = 1;
      ++nlive;
    }
    if (nlive == 0) break;
    for (int q = 0; q < ns; ++q) {
      fac[q] = live[q] ? 1.0 / beta[q] : 0.0;
      k_s[q] = 0;
      std::fill(&g[(size_t)q * (restart + 1)], &g[(size_t)q * (restart + 1)] + restart + 1, 0.0);
      g[(size_t)q * (restart + 1)] = live[q] ? beta[q] : 0.0;
    }
    CU_TRY(cudaMemcpyAsync(dF, fac.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
    airg::note_launch(), k_seg_scale<<<B->seg.nblk, 256, 0, s>>>(B->r, B->V, B->seg, dF);
    std::vector<int> going = live;
    int j = 0;
    for (; j < restart; ++j) {
      double* vj = B->V + (size_t)j * N;
      double* zj = B->Zk + (size_t)j * N;
      CU_TRY(cudaMemcpyAsync(B->gin, vj, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      CU_TRY(cudaGraphLaunch(B->vg, s));
      g_launches.fetch_add(B->vg_kernels);
      CU_TRY(cudaMemcpyAsync(zj, B->gout, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      AIRG_TRY(spmv_mapped(B->A0, zj, nullptr, B->w, SPMV_SET, s));
      AIRG_TRY(seg_gs(B, B->V, j + 1, B->w, nullptr, dH1, nullptr));
      AIRG_TRY(seg_gs(B, B->V, j + 1, B->w, dH1, dH2, nullptr));
      AIRG_TRY(seg_gs(B, B->V, j + 1, B->w, dH2, nullptr, dN));
      AIRG_TRY(read());
      int ngoing = 0;
      for (int q = 0; q < ns; ++q) {
        fac[q] = 0.0;
        if (!going[q]) continue;
        double* h = &Hh[((size_t)q * restart + j) * (restart + 1)];
        for (int i = 0; i <= j; ++i) h[i] = hH1[(size_t)q * CS + i] + hH2[(size_t)q * CS + i];
        const double hj1 = std::sqrt(hN[q]);
        h[j + 1] = hj1;
        double* c_ = &cs[(size_t)q * restart];
        double* s_ = &sn[(size_t)q * restart];
        double* gq = &g[(size_t)q * (restart + 1)];
        for (int i = 0; i < j; ++i) {
          const double t1 = h[i], t2 = h[i + 1];
          h[i] = c_[i] * t1 + s_[i] * t2;
          h[i + 1] = -s_[i] * t1 + c_[i] * t2;
        }
        const double dd = std::hypot(h[j], h[j + 1]);
        double cc = 1.0, ss = 0.0;
        if (dd != 0.0) { cc = h[j] / dd; ss = h[j + 1] / dd; }
        h[j] = cc * h[j] + ss * h[j + 1];
        h[j + 1] = 0.0;
        c_[j] = cc;
        s_[j] = ss;
        gq[j + 1] = -ss * gq[j];
        gq[j] = cc * gq[j];
        iters[q]++;
        k_s[q] = j + 1;
        const double est = std::fabs(gq[j + 1]) / bn[q];
        if (est <= o->rtol || hj1 == 0.0 || !(est == est) || iters[q] >= o->max_it) {
          going[q] = 0;
          continue;
        }
        fac[q] = 1.0 / hj1;
        ++ngoing;
      }
      if (ngoing == 0 || j + 1 == restart) { ++j; break; }
      CU_TRY(cudaMemcpyAsync(dF, fac.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
      airg::note_launch(), k_seg_scale<<<B->seg.nblk, 256, 0, s>>>(B->w, B->V + (size_t)(j + 1) * N, B->seg, dF);
      KERNEL_CHECK();
    }
    for (int q = 0; q < ns; ++q) {
      const int k = live[q] ? k_s[q] : 0;
      cnt[q] = k;
      const double* gq = &g[(size_t)q * (restart + 1)];
      for (int i = k - 1; i >= 0; --i) {
        double t = gq[i];
        for (int p = i + 1; p < k; ++p) t -= Hh[((size_t)q * restart + p) * (restart + 1) + i] * Y[(size_t)q * CS + p];
        Y[(size_t)q * CS + i] = t / Hh[((size_t)q * restart + i) * (restart + 1) + i];
      }
    }
    CU_TRY(cudaMemcpyAsync(dY, Y.data(), sizeof(double) * (size_t)ns * CS, cudaMemcpyHostToDevice, s));
    CU_TRY(cudaMemcpyAsync(B->dcnt, cnt.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    airg::note_launch(), k_seg_axpy<<<B->seg.nblk, 256, 0, s>>>(B->Zk, N, B->xp, B->seg, dY, B->dcnt);
    KERNEL_CHECK();
    AIRG_TRY(residual());
  }
  for (int q = 0; q < ns; ++q) {
    airg_hierarchy* H = B->H[q];
    if (H->n0 > 0) airg::note_launch(), k_perm_out<<<grid_for(H->n0, 256), 256, 0, s>>>(B->xp, H->pos0, x[q], B->base[q], H->n0);
    infos[q].iters = iters[q];
    infos[q].relres = relres[q];
    infos[q].status = status[q];
    infos[q].levels = (int)H->lv.size();
  }
  KERNEL_CHECK();
  CU_TRY(cudaStreamSynchronize(s));
  int worst = AIRG_OK;
  for (int q = 0; q < ns; ++q)
    if (status[q] < 0) return status[q];
    else if (status[q] > worst) worst = status[q];
  return worst;
}

}  // extern "C"
