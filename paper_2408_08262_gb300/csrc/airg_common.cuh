// Shared declarations of the AIRG CUDA library (sm_103a).  Device data layout:
//   * CSR operators: int32 row pointers / columns, FP64 values, one allocation per array.
//   * Every level's solve-phase vectors live in ONE nested buffer per role: level l's vector
//     occupies [off_l, off_l + n_l) with off_{l+1} = off_l + n_f(l), because level l stores its
//     unknowns F-points first and its C-points (= level l+1's unknowns, in level l+1's own F-then-C
//     order) last.  Restriction, recursion and prolongation therefore never permute.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/airg.h"

namespace airg {

#define AIRG_TRY(expr)          \
  do {                          \
    int _rc = (expr);           \
    if (_rc != AIRG_OK) return _rc; \
  } while (0)

inline int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return AIRG_OK;
  if (e == cudaErrorMemoryAllocation) return AIRG_ERR_OOM;
  return AIRG_ERR_CUDA;
}
#define CU_TRY(expr) AIRG_TRY(::airg::cuda_status(expr))
#define KERNEL_CHECK() CU_TRY(cudaGetLastError())

constexpr int kF = 1;  // CF marker values (device and export): 0 unassigned, 1 F, 2 C
constexpr int kC = 2;

// Library-owned device CSR.
// Sliced ELL copy of a CSR operator for the solve (FP64): rows sorted by length within windows of
// kSellWindow rows, then cut into slices of 32 rows; slice s holds its rows' entries column-major
// (entry k of the slice's lane l at sp[s] + 32 k + l), padded to the slice's longest row with
// column -1.  perm[32 s + l] is the CSR row of that lane (-1 past the last row).  Entries keep their
// CSR order within a row.
struct DSell {
  int nrows = 0, nslices = 0;
  long long nnz_pad = 0;
  int* sp = nullptr;
  int* ci = nullptr;
  double* v = nullptr;
  int* perm = nullptr;
  void* v_lo = nullptr;  // the values as float (vt 1) or bf16 (vt 2) for the mixed-precision V-cycle
  int vt = 0;
};
constexpr int kSellWindow = 1024;

struct DCsr {
  int nrows = 0, ncols = 0, nnz = 0;
  int* rp = nullptr;
  int* ci = nullptr;
  double* v = nullptr;
  const DSell* sell = nullptr;  // optional sliced ELL copy the FP64 SpMVs use instead (solve operators)
};

// Stream-ordered device memory.  An Arena hands out 256-byte-aligned sub-ranges of large chunks
// obtained with cudaMallocAsync (bump allocation), so a hierarchy owns a handful of blocks rather
// than thousands of arrays.  reset() makes every chunk reusable (all users are on the same stream,
// so later kernels see the memory only after earlier ones are done); release() frees the chunks.
struct Arena {
  cudaStream_t s = nullptr;
  size_t chunk_min = (size_t)64 << 20;
  bool no_grow = false;  // true: only the chunks given up front are used (no device allocation)
  struct Chunk {
    char* base;
    size_t size, used;
  };
  std::vector<Chunk> chunks;
  size_t cur = 0;  // first chunk that may still have room
  template <class T>
  int alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    const size_t bytes = ((n * sizeof(T)) + 255) & ~(size_t)255;
    for (size_t c = cur; c < chunks.size(); ++c) {
      if (chunks[c].size - chunks[c].used >= bytes) {
        *p = reinterpret_cast<T*>(chunks[c].base + chunks[c].used);
        chunks[c].used += bytes;
        return AIRG_OK;
      }
      if (c == cur && chunks[c].size - chunks[c].used < 4096) ++cur;  // nearly full: skip from now on
    }
    if (no_grow) return AIRG_ERR_SCRATCH;
    size_t sz = bytes > chunk_min ? bytes : chunk_min;
    void* b = nullptr;
    cudaError_t e = cudaMallocAsync(&b, sz, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? AIRG_ERR_OOM : AIRG_ERR_CUDA;
    }
    chunks.push_back({(char*)b, sz, bytes});
    *p = reinterpret_cast<T*>(b);
    return AIRG_OK;
  }
  int csr(DCsr& A, int nrows, int ncols, int nnz) {
    A.nrows = nrows;
    A.ncols = ncols;
    A.nnz = nnz;
    AIRG_TRY(alloc(&A.rp, (size_t)nrows + 1));
    AIRG_TRY(alloc(&A.ci, (size_t)nnz));
    AIRG_TRY(alloc(&A.v, (size_t)nnz));
    return AIRG_OK;
  }
  void reset() {
    for (auto& c : chunks) c.used = 0;
    cur = 0;
  }
  void release() {
    for (auto& c : chunks) cudaFreeAsync(c.base, s);
    chunks.clear();
    cur = 0;
  }
};

// Every kernel launch of the library is counted (airg_launch_count).
extern std::atomic<long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
inline int grid_for(long long work, int block, int cap = 152 * 32) {
  long long g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------------------------------------
// Primitives (airg_prims.cu)
// ------------------------------------------------------------------------------------------
// Exclusive scan of n int32 values into out (n+1 entries, out[n] = total); total also returned
// to *total_host when non-null (synchronises the stream).
int scan_i32(const int* in, int* out, int n, Arena& tmp, cudaStream_t s, long long* total_host);
int scan_i64(const long long* in, long long* out, int n, Arena& tmp, cudaStream_t s, long long* total_host);

// Deterministic FP64 reductions: multi-column dot products and norms, two-stage with a fixed
// grid and the final stage done by the last block to finish.
struct Reducer {
  double* partial = nullptr;  // [kRedBlocks * kRedCols]
  unsigned* counter = nullptr;
};
constexpr int kRedBlocks = 152 * 8;  // 8 CTAs of 256 threads per SM: enough loads in flight for HBM
constexpr int kRedCols = 34;
int reducer_init(Reducer& r, Arena& a, cudaStream_t s);

// out[0] = x.x (n entries)
int dev_nrm2sq(const double* x, int n, double* out, Reducer& r, cudaStream_t s);

// Gram-Schmidt pass over the first ncols columns of V (column-major, leading dim ldv):
//   if hsub: w -= V hsub;   then dots[k] = V_k . w (k < ncols) and, if nrm, nrm[0] = w . w.
int dev_gs_pass(const double* V, long long ldv, int ncols, double* w, int n, const double* hsub, double* dots,
                double* nrm, Reducer& r, cudaStream_t s);

// x += V y (first ncols columns)
int dev_multi_axpy(const double* V, long long ldv, int ncols, const double* y, double* x, int n, cudaStream_t s);

// SpMV epilogues
enum SpmvMode { SPMV_SET = 0, SPMV_RESID = 1, SPMV_ADD = 2, SPMV_ADDB = 3, SPMV_AXPB = 4 };
// y = A x (SET) | b - A x (RESID) | y + A x (ADD) | b + A x (ADDB; y may alias b)
int dev_spmv(const DCsr& A, const double* x, const double* b, double* y, int mode, int lanes, cudaStream_t s);
// Sliced ELL copies of solve operators (airg_sell.cu).  want_sell: large operators with short rows.
// build_sell synchronises the stream (the padded size allocates the arrays).  sell_spmv: the same
// modes and epilogues as the CSR SpMVs (w != nullptr: RESID with the fused one-point prolongation).
constexpr int kSellMinRows = 32768;
bool want_sell(const DCsr& A);
int build_sell(const DCsr& A, DSell& out, Arena& own, Arena& tmp, cudaStream_t s);
int sell_spmv(const DSell& S, const double* x, const double* b, double* y, int mode, const int* w, double* xf,
              const double* coef, cudaStream_t s);
// Mixed precision: the copy's values cast to float (vt 1) or bf16 (vt 2); the SpMV with float
// vectors and accumulation (the same modes, w != nullptr: RESID with the fused prolongation).
int sell_cast_values(DSell& S, int vt, Arena& own, cudaStream_t s);
int sell_spmv_lo(const DSell& S, const float* x, const float* b, float* y, int mode, const int* w, float* xf,
                 cudaStream_t s);
// y = coef[0] r, or y += coef[0] r with add (coef on the device); x += y
void dev_coef_axpy(const double* coef, const double* r, double* y, int n, bool add, cudaStream_t s);
void dev_add(const double* y, double* x, int n, cudaStream_t s);
// y = coef[0] b + A x, coef a device scalar
int dev_spmv_axpb(const DCsr& A, const double* x, const double* b, const double* coef, double* y, int lanes,
                  cudaStream_t s);
int pick_lanes(double avg_row_len);
// Solve operators whose arrays take at most this many MiB are read with the evict-normal L2
// policy (AIRG_L2_KEEP_MB overrides; l2_keep_bytes gives the size in bytes), larger ones with
// evict-first.
constexpr int kL2KeepMB = 64;
double l2_keep_bytes();
#ifdef __CUDACC__
// Loads of an operator's columns and values with an L2 eviction policy held in a register:
// evict-first for operators that stream through L2 once per use (they would only displace the
// vectors), evict-normal for operators small enough that the level's second smoothing pass and
// the coarsest level's iterations find them still in L2.
__device__ __forceinline__ uint64_t l2_policy(bool keep) {
  uint64_t p;
  if (keep) asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  else asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_pol(const int* p, uint64_t pol) {
  int v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_pol(const double* p, uint64_t pol) {
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_pol(const float* p, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ __nv_bfloat16 ld_pol(const __nv_bfloat16* p, uint64_t pol) {
  unsigned short v;
  asm("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return __ushort_as_bfloat16(v);
}
#endif
// r = b_F - AF x with x_F taken as the one-point prolongation of x_C (x[f] = x[nf + w[f]]), which
// is also stored into x_F.  AF has nf rows; x holds [x_F, x_C].
int dev_spmv_resid_prolong(const DCsr& AF, double* x, const int* w, const double* b, double* y, int lanes,
                           cudaStream_t s);

// Mixed-precision V-cycle: values float (vt 1) or bf16 (vt 2), vectors/accumulation float.
int dev_spmv_lo(const DCsr& A, const void* vals, int vt, const float* x, const float* b, float* y, int mode, int lanes,
                const int* w, cudaStream_t s);
void dev_cast_d2f(const double* in, float* out, long long n, cudaStream_t s);
void dev_cast_d2bf(const double* in, void* out, long long n, cudaStream_t s);
void dev_cast_f2d(const float* in, double* out, long long n, cudaStream_t s);
void dev_gather_prolong_f(float* x, int nf, const int* w, cudaStream_t s);

void dev_scale(const double* x, double alpha_div, double* y, int n, cudaStream_t s);  // y = x * (1 / a)
void dev_permute(const double* in, const int* pos, double* out, int n, bool inverse, cudaStream_t s);
void dev_gather_prolong(double* x, int nf, const int* w, cudaStream_t s);  // x[f] = x[nf + w[f]]
void dev_fill(double* x, double v, int n, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Setup (airg_setup.cu)
// ------------------------------------------------------------------------------------------
struct SetupParams {
  double strong_threshold, ddc_fraction, drop_R, drop_Ac;
  int pmisr_max_loops, poly_order, coarse_poly_order, coarse_iters, coarse_size, max_levels, n_smooth_up;
  uint64_t seed;
  int sparsity_order = 1;  // fixed sparsity of the A_ff polynomials: 1 pattern(A_ff), 2 pattern(A_ff^2)
  int ideal_prolong = 0;   // 1: P = [W; I] with W = -Ainv A_fc (drop_R), else one-point
  // re-used CF splittings: cf_reuse[l] (device int8, level l's size) replaces the split of level l
  // for l < n_reuse
  std::vector<const int8_t*> cf_reuse;
};

// theta_i = sum_{j in F, j != i} |a_ij| / |a_ii| for the F-points of cf (0 for C-points), the
// quantity DDC ranks (Algorithm 2).
int ddc_theta(const DCsr& A, const int8_t* cf, double* theta, Arena& tmp, cudaStream_t s);

// Level l's splitting taken from elsewhere (setup re-use): copies cf_in, computes the strength
// flags the one-point prolongator needs, and counts the F-points (synchronises the stream).
int reuse_split(const DCsr& A, const SetupParams& p, const int8_t* cf_in, int8_t* cf, uint8_t* strong, int* nf_out,
                Arena& tmp, cudaStream_t s);

// CF splitting of A (natural numbering); cf: device int8 n (1 F, 2 C).  strong (device uint8 nnz)
// receives the strength flags when non-null.  nf_out: number of F-points.
int cf_split(const DCsr& A, const SetupParams& p, int level, int8_t* cf, uint8_t* strong, int* nf_out,
             Arena& tmp, cudaStream_t s);

// GMRES polynomial coefficients of A (m coefficients) from the Box-Muller rhs of (seed, level).
// alpha: device m doubles; fitted: device int (number of coefficients fitted before a breakdown).
int poly_fit(const DCsr& A, int m, uint64_t seed, int level, double* alpha, int* fitted, Arena& tmp,
             cudaStream_t s);

// Fixed-sparsity approximate inverse on the pattern of A (order 1) or of A^2 (order 2); A must store
// its diagonal.
int fixed_sparsity_inverse(const DCsr& A, const double* alpha, int m, DCsr& out, Arena& own, Arena& tmp,
                           cudaStream_t s, int order);

// C = scale * (A B) with the relative row-wise inf-norm drop (|c| < tol max|c_i.| dropped; the
// diagonal kept when keep_diag).
// Sparse product in padded form: row i's cnt[i] entries (sorted columns) at tcol/tval + ubo[i].
struct SpgPadded {
  int nrows = 0, ncols = 0;
  long long total = 0;       // candidate slots
  long long* ubo = nullptr;  // nrows + 1 slot offsets
  int* beg = nullptr;        // the offsets as int (nullptr when total exceeds int range)
  int* cnt = nullptr;
  int* tcol = nullptr;
  double* tval = nullptr;
  int* err = nullptr;        // device flag: a row exceeded the block path's capacity
};
int spgemm_padded(const DCsr& A, const DCsr* Bc, const SpgPadded* Bp, double scale, double tol, bool keep_diag,
                  SpgPadded& out, Arena& tmp, cudaStream_t s);
int spgemm_compact(const SpgPadded& P, DCsr& out, Arena& own, Arena& tmp, cudaStream_t s);
int spgemm(const DCsr& A, const DCsr& B, double scale, double tol, bool keep_diag, DCsr& out, Arena& own,
           Arena& tmp, cudaStream_t s);

struct LevelBuild {
  // natural-numbering setup data of one level (owned by `own`)
  DCsr A;            // level matrix
  int n = 0, nf = 0, nc = 0;
  int8_t* cf = nullptr;
  int* pos = nullptr;   // natural index -> F-then-C position
  int* Fnat = nullptr;  // F index -> natural
  int* Cnat = nullptr;  // C index -> natural
  DCsr Aff, Afc, Acf, Ainv, Z;
  DCsr W;               // approximate ideal prolongator (n_f x n_c, natural C numbering); empty for one-point
  int* w = nullptr;     // F index -> C index (natural C numbering), -1 none
  double* alpha = nullptr;
  int m = 0, fitted = 0;
  int* fitted_dev = nullptr;  // device copy of `fitted`, read back once the hierarchy is built
  bool coarsest = false;
  // phase boundaries (CUDA events, recorded when non-null): start, CF split, extraction,
  // polynomial (steps 3-8), restrictor, prolongator + coarse matrix
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};

// A second stream for work of a level that does not depend on the polynomial (the one-point
// prolongator and A P), with its own scratch arena and two events (fork, join).
struct SideStream {
  cudaStream_t s = nullptr;
  Arena* tmp = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// Builds level data and the next coarse matrix (setup steps 1-11).  If the level turns out to be
// the coarsest, only the polynomial is built and *Ac_out is left empty.  With `side`, the one-point
// prolongator and A P run on the side stream while the polynomial is fitted on s.
int build_level(const DCsr& A, const SetupParams& p, int level, bool force_coarsest, LevelBuild& L,
                DCsr& Ac_out, Arena& own, Arena& tmp, cudaStream_t s, const SideStream* side = nullptr);

// Nested solve numbering of a non-coarsest level from its F/C positions and the next level's
// nested numbering (nullptr when the next level is the coarsest: identity there).
int compose_layout(const LevelBuild& L, const int* lay_next, int* lay, cudaStream_t s);
// Solve-phase operators of level l given level l+1's nested numbering (nullptr: identity).
int build_solve_ops(const LevelBuild& L, const int* pos_next, DCsr& AF, DCsr& Zs, int** ws, DCsr& Ws, Arena& own,
                    Arena& tmp, cudaStream_t s);
// Symmetric permutation of A by pos: row pos[i] gets row i with columns pos[j].
int permute_matrix(const DCsr& A, const int* pos, DCsr& out, Arena& own, Arena& tmp, cudaStream_t s);

// Input validation: sorted unique in-range columns, nonzero diagonal.
int validate_csr(const DCsr& A, Arena& tmp, cudaStream_t s);

// Host-side argument checks of the entry points (airg_api.cu): null pointers, negative sizes and
// parameters outside their ranges give AIRG_ERR_ARG before any device work.
int check_params(const airg_params* p);
int check_csr_arg(const airg_csr* A);

}  // namespace airg
