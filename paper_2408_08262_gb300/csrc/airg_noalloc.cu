// CF splitting without any device allocation.
//
// Some callers cannot allocate device memory once they are running: a host program that reserves
// all of its GPU memory up front and hands out only what it pre-reserved, a solver embedded in a
// real-time or latency-critical loop where an allocation (and the synchronisation it may cause) is
// not acceptable, or code that runs while a framework's allocator owns the device.  For them,
// airg_cf_split_noalloc computes exactly what airg_cf_split computes, but every temporary lives in
// the fixed array below, which the library reserves when it is loaded on a device.
#include <mutex>

#include "airg_common.cuh"

namespace airg {

// Capacity of the scratch array: 32 MiB on every GPU that loads the library, held until the
// process exits.  A matrix needs about 5 bytes per nonzero plus 34 bytes per row (see
// noalloc_need); larger inputs are rejected with AIRG_ERR_SCRATCH before any GPU work.
constexpr size_t kNoAllocBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_cf_scratch[kNoAllocBytes];

namespace {
std::mutex g_mu;
void* g_ptr[256] = {};  // device address of g_cf_scratch, per device ordinal

// Upper bound of the scratch the CF splitting takes for an n x n matrix with nnz nonzeros: strength
// flags (1 B/nnz), transposed strong lists (4 B/nnz), five int arrays and two double arrays over the
// rows, one byte per row, scan tile sums and alignment slack.
size_t noalloc_need(long long n, long long nnz) { return (size_t)(5 * nnz + 34 * n + 65536); }

// Host-side address of the array on the current device (looked up once per device).
int scratch_ptr(void** out) {
  int dev = 0;
  CU_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return AIRG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_cf_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return AIRG_ERR_CUDA;
    }
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return AIRG_OK;
}
}  // namespace

}  // namespace airg

using namespace airg;

extern "C" int airg_cf_split_noalloc(const airg_csr* A, const airg_params* p, int level, int8_t* cf_out,
                                     airg_stream_t stream) {
  if (!A || !p || !cf_out || level < 0 || A->n < 0 || A->nnz < 0) return AIRG_ERR_ARG;
  if (noalloc_need(A->n, A->nnz) > kNoAllocBytes) return AIRG_ERR_SCRATCH;
  if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val)))) return AIRG_ERR_ARG;
  if (!(p->strong_threshold >= 0.0 && p->strong_threshold <= 1.0)) return AIRG_ERR_ARG;
  if (!(p->ddc_fraction >= 0.0 && p->ddc_fraction <= 1.0)) return AIRG_ERR_ARG;
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
