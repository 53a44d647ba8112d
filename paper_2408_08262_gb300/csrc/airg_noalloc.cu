// CF splitting without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a host program that reserves
// all of its GPU memory up front and hands out only what it pre-reserved, a solver embedded in a
// real-time or latency-critical loop where an allocation (and the synchronisation it may cause) is
// not acceptable, or code that runs while a framework's allocator owns the device.  For them,
// airg_cf_split_noalloc computes exactly what airg_cf_split computes, but every temporary lives in
// the fixed array below.  CUDA loads a module (its kernels and its __device__ arrays) lazily, on
// first use: the array is allocated on a device by the first call made there, which also loads the
// kernels the splitting launches.  That first call therefore allocates; later calls do not.
#include <mutex>
#include <vector>

#include "airg_common.cuh"

namespace airg {

// Capacity of the scratch array: 32 MiB on every GPU on which the entry point has been called,
// held until the process exits.  A matrix needs about 5 bytes per nonzero plus 34 bytes per row (see
// noalloc_need); larger inputs are rejected with AIRG_ERR_SCRATCH before any GPU work.
constexpr size_t kNoAllocBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_cf_scratch[kNoAllocBytes];

namespace {
std::mutex g_mu;

// Upper bound of the scratch the CF splitting takes for an n x n matrix with nnz nonzeros: strength
// flags (1 B/nnz), transposed strong lists (4 B/nnz), five int arrays and two double arrays over the
// rows, one byte per row, scan tile sums and alignment slack.
size_t noalloc_need(long long n, long long nnz) { return (size_t)(5 * nnz + 34 * n + 65536); }

// The array's device address, looked up once per device and context.  A context is identified by
// its process-unique id (cuCtxGetId), so a context created anew on a device (after cudaDeviceReset,
// for example) looks the address up again instead of reusing one that pointed into the old context.
// The two driver calls are reached through the runtime's entry-point query, so the library does not
// link the driver library itself.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
struct CachedAddr {
  int dev;
  unsigned long long ctx_id;
  void* ptr;
};
std::vector<CachedAddr> g_cache;
CtxGetCurrentFn g_get_ctx = nullptr;
CtxGetIdFn g_get_id = nullptr;
bool g_fns_looked_up = false;

// Id of the current context, or false when it cannot be determined (then nothing is cached).
bool current_ctx_id(unsigned long long* id) {
  if (!g_fns_looked_up) {
    g_fns_looked_up = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      g_get_ctx = (CtxGetCurrentFn)f1;
      g_get_id = (CtxGetIdFn)f2;
    }
    cudaGetLastError();
  }
  if (!g_get_ctx || !g_get_id) return false;
  void* ctx = nullptr;
  if (g_get_ctx(&ctx) != 0 || !ctx) return false;
  return g_get_id(ctx, id) == 0;
}

// Set-up: the array's device address for the current device and context (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
int scratch_ptr(void** out) {
  int dev = 0;
  CU_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  if (current_ctx_id(&id))
    for (const CachedAddr& c : g_cache)
      if (c.dev == dev && c.ctx_id == id) {
        *out = c.ptr;
        return AIRG_OK;
      }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_cf_scratch);  // loads the module on first use
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AIRG_ERR_CUDA;
  }
  if (current_ctx_id(&id)) g_cache.push_back({dev, id, p});
  *out = p;
  return AIRG_OK;
}
}  // namespace

}  // namespace airg

using namespace airg;

extern "C" int airg_cf_split_noalloc(const airg_csr* A, const airg_params* p, int level, int8_t* cf_out,
                                     airg_stream_t stream) {
  // the argument checks of airg_cf_split, then the capacity
  AIRG_TRY(check_csr_arg(A));
  AIRG_TRY(check_params(p));
  if (!cf_out || level < 0) return AIRG_ERR_ARG;
  if (noalloc_need(A->n, A->nnz) > kNoAllocBytes) return AIRG_ERR_SCRATCH;
  void* base = nullptr;
  AIRG_TRY(scratch_ptr(&base));
  cudaStream_t s = (cudaStream_t)stream;
  // an arena over the fixed array: it never allocates, it fails once the array is full
  Arena fixed;
  fixed.s = s;
  fixed.no_grow = true;
  fixed.chunks.push_back({(char*)base, kNoAllocBytes, 0});
  DCsr D;
  D.nrows = D.ncols = A->n;
  D.nnz = A->nnz;
  D.rp = const_cast<int*>(A->rowptr);
  D.ci = const_cast<int*>(A->col);
  D.v = const_cast<double*>(A->val);
  SetupParams sp;
  sp.strong_threshold = p->strong_threshold;
  sp.ddc_fraction = p->ddc_fraction;
  sp.drop_R = p->drop_R;
  sp.drop_Ac = p->drop_Ac;
  sp.pmisr_max_loops = p->pmisr_max_loops;
  sp.poly_order = p->poly_order;
  sp.coarse_poly_order = p->coarse_poly_order;
  sp.coarse_iters = p->coarse_iters;
  sp.coarse_size = p->coarse_size;
  sp.max_levels = p->max_levels;
  sp.n_smooth_up = p->n_smooth_up;
  sp.seed = p->seed;
  int rc = validate_csr(D, fixed, s);
  int nf = 0;
  if (rc == AIRG_OK) rc = cf_split(D, sp, level, cf_out, nullptr, &nf, fixed, s);
  if (rc == AIRG_OK) rc = cuda_status(cudaStreamSynchronize(s));
  return rc;
}
