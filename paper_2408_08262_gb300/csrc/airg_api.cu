// C ABI of libairg.so (declared in include/airg.h): hierarchy construction, solves, CF-splitting
// and export hooks, kernel timing.
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <vector>
#include <atomic>
#include <thread>
#include <new>

#include "airg_hier.cuh"

using namespace airg;

namespace airg {
std::atomic<long long> g_launches{0};

}

namespace {

SetupParams to_setup(const airg_params& p) {
  SetupParams q;
  q.strong_threshold = p.strong_threshold;
  q.ddc_fraction = p.ddc_fraction;
  q.drop_R = p.drop_R;
  q.drop_Ac = p.drop_Ac;
  q.pmisr_max_loops = p.pmisr_max_loops;
  q.poly_order = p.poly_order;
  q.coarse_poly_order = p.coarse_poly_order;
  q.coarse_iters = p.coarse_iters;
  q.coarse_size = p.coarse_size;
  q.max_levels = p.max_levels;
  q.n_smooth_up = p.n_smooth_up;
  q.seed = p.seed;
  q.sparsity_order = p.sparsity_order;
  q.ideal_prolong = p.ideal_prolong;
  return q;
}

// Algorithmic bytes of one SpMV with the given epilogue: the CSR arrays once, x once per column
// (every solve operator references essentially all of its columns), y written once, and b
// (RESID/ADDB) or y (ADD) read once.
double spmv_bytes(const DCsr& A, bool reads_extra, double vb = 8.0, double xb = 8.0) {
  return (vb + 4.0) * A.nnz + 4.0 * (A.nrows + 1) + xb * A.ncols + xb * A.nrows * (reads_extra ? 2 : 1);
}

// Mixed precision: copies of the V-cycle operators' values in float (vt 1) or bf16 (vt 2).
int cast_values(const DCsr& A, int vt, void** out, Arena& a, cudaStream_t s) {
  if (vt == 1) {
    float* p;
    AIRG_TRY(a.alloc(&p, std::max(A.nnz, 1)));
    dev_cast_d2f(A.v, p, A.nnz, s);
    *out = p;
  } else {
    uint16_t* p;
    AIRG_TRY(a.alloc(&p, std::max(A.nnz, 1)));
    dev_cast_d2bf(A.v, p, A.nnz, s);
    *out = p;
  }
  CU_TRY(cudaGetLastError());
  return AIRG_OK;
}

int copy_csr(const DCsr& A, DCsr& B, Arena& a, cudaStream_t s) {
  AIRG_TRY(a.csr(B, A.nrows, A.ncols, A.nnz));
  CU_TRY(cudaMemcpyAsync(B.rp, A.rp, sizeof(int) * ((size_t)A.nrows + 1), cudaMemcpyDeviceToDevice, s));
  CU_TRY(cudaMemcpyAsync(B.ci, A.ci, sizeof(int) * (size_t)A.nnz, cudaMemcpyDeviceToDevice, s));
  CU_TRY(cudaMemcpyAsync(B.v, A.v, sizeof(double) * (size_t)A.nnz, cudaMemcpyDeviceToDevice, s));
  return AIRG_OK;
}

double avg_len(const DCsr& A) { return A.nrows > 0 ? (double)A.nnz / A.nrows : 1.0; }

// Matrix-free form: the level's coefficients (and A_ff, off the coarsest level) in solve memory.
static int keep_polynomial(const LevelBuild& L, SolveLevel& S, Arena& a, cudaStream_t s) {
  S.m = L.m;
  if (L.m > 0) {
    AIRG_TRY(a.alloc(&S.alpha, L.m));
    CU_TRY(cudaMemcpyAsync(S.alpha, L.alpha, sizeof(double) * (size_t)L.m, cudaMemcpyDeviceToDevice, s));
  }
  if (!L.coarsest) {
    AIRG_TRY(copy_csr(L.Aff, S.Aff, a, s));
    S.lanes_Aff = pick_lanes(avg_len(S.Aff));
  }
  return AIRG_OK;
}

int setup_impl(airg_hierarchy* H, const airg_csr* Ain, const airg_hierarchy* T, int reuse_levels, bool host_input) {
  cudaStream_t s = H->s;
  SetupParams sp = to_setup(H->p);
  if (sp.coarse_size <= 0) sp.coarse_size = (int)std::min<long long>(60000, std::max<long long>(64, (long long)Ain->n / 16));
  if (T) {  // setup re-use: the template's splittings for its leading non-coarsest levels
    const int avail = (int)T->lv.size() - 1;
    const int k = reuse_levels <= 0 ? avail : std::min(reuse_levels, avail);
    for (int l = 0; l < k; ++l) sp.cf_reuse.push_back(T->lv[l].cf);
  }
  Arena tmp;
  tmp.s = s;
  struct Rel {
    Arena& a;
    ~Rel() { a.release(); }
  } rel{tmp};
  DCsr A0;
  AIRG_TRY(H->setup_mem.csr(A0, Ain->n, Ain->n, Ain->nnz));
  const cudaMemcpyKind kind = host_input ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CU_TRY(cudaMemcpyAsync(A0.rp, Ain->rowptr, sizeof(int) * ((size_t)Ain->n + 1), kind, s));
  CU_TRY(cudaMemcpyAsync(A0.ci, Ain->col, sizeof(int) * (size_t)Ain->nnz, kind, s));
  CU_TRY(cudaMemcpyAsync(A0.v, Ain->val, sizeof(double) * (size_t)Ain->nnz, kind, s));
  AIRG_TRY(validate_csr(A0, tmp, s));
  H->n0 = Ain->n;
  H->top_nnz = Ain->nnz;
  DCsr A = A0;
  std::vector<cudaEvent_t> evs;
  struct EvRel {
    std::vector<cudaEvent_t>& v;
    ~EvRel() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } evrel{evs};
  Arena lt;  // per-level scratch, reset and reused level after level
  lt.s = s;
  lt.chunk_min = (size_t)256 << 20;
  struct LtRel {
    Arena& a;
    ~LtRel() { a.release(); }
  } ltrel{lt};
  // side stream for the work of a level that does not wait for its polynomial
  Arena lt2;
  lt2.chunk_min = (size_t)256 << 20;
  SideStream side;
  side.tmp = &lt2;
  struct SideRel {
    SideStream& sd;
    Arena& a;
    ~SideRel() {
      if (sd.s) cudaStreamSynchronize(sd.s);
      a.release();
      if (sd.s) cudaStreamSynchronize(sd.s);
      if (sd.fork) cudaEventDestroy(sd.fork);
      if (sd.join) cudaEventDestroy(sd.join);
      if (sd.s) cudaStreamDestroy(sd.s);
    }
  } siderel{side, lt2};
  if (cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (side.s) cudaStreamDestroy(side.s);
    side.s = nullptr;  // run everything on s
  }
  lt2.s = side.s ? side.s : s;
  for (int l = 0;; ++l) {
    LevelBuild L;
    for (int k = 0; k < 6; ++k)
      if (cudaEventCreate(&L.ev[k]) == cudaSuccess) evs.push_back(L.ev[k]);
      else { L.ev[k] = nullptr; cudaGetLastError(); }
    DCsr Ac;
    lt.reset();
    lt2.reset();
    int rc = build_level(A, sp, l, l == sp.max_levels - 1, L, Ac, H->setup_mem, lt, s, side.s ? &side : nullptr);
    if (rc != AIRG_OK) return rc;
    H->lb.push_back(L);
    if (L.coarsest) break;
    A = Ac;
  }
  cudaEvent_t ev_layout0 = nullptr, ev_layout1 = nullptr;
  if (cudaEventCreate(&ev_layout0) == cudaSuccess) evs.push_back(ev_layout0);
  if (cudaEventCreate(&ev_layout1) == cudaSuccess) evs.push_back(ev_layout1);
  if (ev_layout0) cudaEventRecord(ev_layout0, s);
  // solve-phase operators
  const int nl = (int)H->lb.size();
  H->lv.resize(nl);
  // nested numberings, from the coarsest level upwards
  for (int l = nl - 2; l >= 0; --l) {
    const int* lay_next = (l + 1 < nl - 1) ? H->lv[l + 1].lay : nullptr;
    AIRG_TRY(H->solve_mem.alloc(&H->lv[l].lay, std::max(H->lb[l].n, 1)));
    AIRG_TRY(compose_layout(H->lb[l], lay_next, H->lv[l].lay, s));
  }
  long long off = 0;
  for (int l = 0; l < nl; ++l) {
    LevelBuild& L = H->lb[l];
    SolveLevel& S = H->lv[l];
    S.n = L.n;
    S.off = off;
    S.coarsest = L.coarsest;
    if (L.coarsest) {
      AIRG_TRY(copy_csr(L.A, S.A, H->solve_mem, s));
      AIRG_TRY(copy_csr(L.Ainv, S.Ainv, H->solve_mem, s));
      S.lanes_A = pick_lanes(avg_len(S.A));
      S.lanes_Ainv = pick_lanes(avg_len(S.Ainv));
      if (H->p.matrix_free) AIRG_TRY(keep_polynomial(L, S, H->solve_mem, s));
      break;
    }
    S.nf = L.nf;
    S.nc = L.nc;
    AIRG_TRY(H->solve_mem.alloc(&S.cf, std::max(L.n, 1)));
    CU_TRY(cudaMemcpyAsync(S.cf, L.cf, (size_t)L.n, cudaMemcpyDeviceToDevice, s));
    const int* lay_next = (l + 1 < nl - 1) ? H->lv[l + 1].lay : nullptr;
    AIRG_TRY(build_solve_ops(L, lay_next, S.AF, S.Z, &S.w, S.W, H->solve_mem, tmp, s));
    if (S.W.nrows > 0) S.lanes_W = pick_lanes(avg_len(S.W));
    AIRG_TRY(copy_csr(L.Ainv, S.Ainv, H->solve_mem, s));
    S.lanes_AF = pick_lanes(avg_len(S.AF));
    S.lanes_Ainv = pick_lanes(avg_len(S.Ainv));
    S.lanes_Z = pick_lanes(avg_len(S.Z));
    if (H->p.matrix_free) AIRG_TRY(keep_polynomial(L, S, H->solve_mem, s));
    off += L.nf;
  }
  // top-level operator in the nested solve numbering of level 0
  if (!H->lb[0].coarsest) {
    H->pos0 = H->lv[0].lay;
    AIRG_TRY(permute_matrix(A0, H->pos0, H->A0s, H->solve_mem, tmp, s));
  } else {
    AIRG_TRY(copy_csr(A0, H->A0s, H->solve_mem, s));
    H->pos0 = nullptr;
  }
  H->lanes_A0 = pick_lanes(avg_len(H->A0s));
  // sliced ELL copies of the large short-row FP64 operators whose rows hold about 5 entries or
  // more: the top-level operator and, when the V-cycle runs in FP64, the smoothing residual's
  // [A_ff A_fc].  The shorter-row Ainv and Z stay CSR: there the permuted output and the lost
  // locality of x between a warp's rows cost more than the coalesced loads gain.
  // AIRG_NO_SELL=1 keeps every SpMV on CSR.
  if (!getenv("AIRG_NO_SELL")) {
    auto mk = [&](DCsr& M) -> int {
      if (!want_sell(M)) return AIRG_OK;
      H->sells.emplace_back();
      AIRG_TRY(build_sell(M, H->sells.back(), H->solve_mem, tmp, s));
      M.sell = &H->sells.back();
      return AIRG_OK;
    };
    AIRG_TRY(mk(H->A0s));
    // [A_ff A_fc] in every precision: the mixed-precision V-cycle reads the copy's values cast to
    // float or bf16
    const int vt_sell = H->p.precision == AIRG_FP32 ? 1 : (H->p.precision == AIRG_BF16_VALUES ? 2 : 0);
    for (auto& S : H->lv)
      if (!S.coarsest) {
        const size_t before = H->sells.size();
        AIRG_TRY(mk(S.AF));
        if (vt_sell && H->sells.size() > before) AIRG_TRY(sell_cast_values(H->sells.back(), vt_sell, H->solve_mem, s));
      }
  }
  if (ev_layout1) cudaEventRecord(ev_layout1, s);
  // mixed-precision form: low-precision copies of every V-cycle operator
  H->vt = H->p.precision == AIRG_FP32 ? 1 : (H->p.precision == AIRG_BF16_VALUES ? 2 : 0);
  if (H->vt)
    for (auto& S : H->lv) {
      AIRG_TRY(cast_values(S.Ainv, H->vt, &S.lo_Ainv, H->solve_mem, s));
      if (S.coarsest) {
        AIRG_TRY(cast_values(S.A, H->vt, &S.lo_A, H->solve_mem, s));
      } else {
        AIRG_TRY(cast_values(S.AF, H->vt, &S.lo_AF, H->solve_mem, s));
        AIRG_TRY(cast_values(S.Z, H->vt, &S.lo_Z, H->solve_mem, s));
      }
    }
  // complexities (Section "Strong tolerances"; storage complexity eq. mat_store)
  double gs = 0, os = 0, st = 0;
  for (int l = 0; l < nl; ++l) {
    const LevelBuild& L = H->lb[l];
    gs += L.n;
    os += L.A.nnz;
    // the matrix-free form stores no inverse: its polynomials reuse A_ff and the coarsest A
    const double inv = H->p.matrix_free ? 0.0 : (double)L.Ainv.nnz;
    if (L.coarsest) st += inv + ((H->p.coarse_iters > 1 || H->p.matrix_free) ? L.A.nnz : 0);
    else
      st += inv + L.Aff.nnz + L.Afc.nnz + (L.Z.nnz + (double)L.nc) +
            ((double)L.nc + (L.W.nrows > 0 ? (double)L.W.nnz : (double)L.nf));
  }
  // the prolongator count above is an upper bound (F rows without a C neighbour have no entry)
  H->grid_cx = H->n0 > 0 ? gs / H->n0 : 0;
  H->op_cx = H->top_nnz > 0 ? os / H->top_nnz : 0;
  H->storage_cx = H->top_nnz > 0 ? st / H->top_nnz : 0;
  CU_TRY(cudaStreamSynchronize(s));
  H->phase_ms.assign(nl, std::vector<float>(5, 0.f));
  for (int l = 0; l < nl; ++l)
    for (int k = 0; k < 5; ++k) {
      const LevelBuild& L = H->lb[l];
      float ms = 0.f;
      if (L.ev[k] && L.ev[k + 1] && cudaEventElapsedTime(&ms, L.ev[k], L.ev[k + 1]) == cudaSuccess) H->phase_ms[l][k] = ms;
      cudaGetLastError();
    }
  for (auto& L : H->lb)
    for (auto& e : L.ev) e = nullptr;
  {
    float ms = 0.f;
    if (ev_layout0 && ev_layout1 && cudaEventElapsedTime(&ms, ev_layout0, ev_layout1) == cudaSuccess) H->layout_ms = ms;
    cudaGetLastError();
  }
  for (auto& L : H->lb)
    if (L.fitted_dev) CU_TRY(cudaMemcpy(&L.fitted, L.fitted_dev, sizeof(int), cudaMemcpyDeviceToHost));
  H->alphas.resize(nl);
  for (int l = 0; l < nl; ++l) {
    H->alphas[l].assign(H->lb[l].m, 0.0);
    if (H->lb[l].m) CU_TRY(cudaMemcpy(H->alphas[l].data(), H->lb[l].alpha, sizeof(double) * H->lb[l].m, cudaMemcpyDeviceToHost));
  }
  if (!H->p.keep_setup) {
    H->setup_mem.release();
    for (auto& L : H->lb) {
      // keep the sizes for airg_level_info; drop the pointers
      L.A.rp = L.A.ci = nullptr; L.A.v = nullptr;
      L.cf = nullptr; L.pos = L.Fnat = L.Cnat = nullptr; L.w = nullptr;
      L.Aff.rp = L.Aff.ci = nullptr; L.Afc.rp = L.Afc.ci = nullptr; L.Acf.rp = L.Acf.ci = nullptr;
      L.Z.rp = L.Z.ci = nullptr; L.Ainv.rp = L.Ainv.ci = nullptr; L.W.rp = L.W.ci = nullptr; L.W.v = nullptr;
      L.Aff.v = L.Afc.v = L.Acf.v = L.Z.v = L.Ainv.v = nullptr;
      L.alpha = nullptr;
      L.fitted_dev = nullptr;
    }
    H->kept = false;
  } else {
    H->kept = true;
  }
  return AIRG_OK;
}

void destroy(airg_hierarchy* H) {
  if (!H) return;
  cudaStreamSynchronize(H->s);
  H->solve_mem.release();
  H->setup_mem.release();
  cudaStreamSynchronize(H->s);
  if (H->vg_exec) cudaGraphExecDestroy(H->vg_exec);
  if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
  for (auto e : H->prof.pool) cudaEventDestroy(e);
  for (auto e : H->prof.graph_pool) cudaEventDestroy(e);
  if (H->hsc) cudaFreeHost(H->hsc);
  delete H;
}

}  // namespace

namespace airg {

// Host-side argument checks shared by the entry points (nothing is read on the device).
int check_params(const airg_params* p) {
  if (!p) return AIRG_ERR_ARG;
  if (!(p->strong_threshold >= 0.0 && p->strong_threshold <= 1.0)) return AIRG_ERR_ARG;
  if (!(p->ddc_fraction >= 0.0 && p->ddc_fraction <= 1.0)) return AIRG_ERR_ARG;
  if (p->poly_order < 0 || p->poly_order > 14 || p->coarse_poly_order < 0 || p->coarse_poly_order > 14) return AIRG_ERR_ARG;
  if (p->coarse_iters < 1 || p->max_levels < 1 || p->n_smooth_up < 0) return AIRG_ERR_ARG;
  if (!(p->drop_R >= 0.0) || !(p->drop_Ac >= 0.0)) return AIRG_ERR_ARG;
  if (p->precision != AIRG_FP64 && p->precision != AIRG_FP32 && p->precision != AIRG_BF16_VALUES) return AIRG_ERR_ARG;
  if (p->sparsity_order != 1 && p->sparsity_order != 2) return AIRG_ERR_ARG;
  if (p->matrix_free != 0 && p->matrix_free != 1) return AIRG_ERR_ARG;
  if (p->matrix_free && p->precision != AIRG_FP64) return AIRG_ERR_ARG;
  if (p->ideal_prolong != 0 && p->ideal_prolong != 1) return AIRG_ERR_ARG;
  if (p->ideal_prolong && p->precision != AIRG_FP64) return AIRG_ERR_ARG;
  return AIRG_OK;
}

int check_csr_arg(const airg_csr* A) {
  if (!A || A->n < 0 || A->nnz < 0) return AIRG_ERR_ARG;
  if (A->n > 0 && (!A->rowptr || (A->nnz > 0 && (!A->col || !A->val)))) return AIRG_ERR_ARG;
  return AIRG_OK;
}

}  // namespace airg

extern "C" {

void airg_params_default(airg_params* p) {
  if (!p) return;
  p->strong_threshold = 0.5;
  p->ddc_fraction = 0.1;
  p->pmisr_max_loops = 3;
  p->poly_order = 6;
  p->coarse_poly_order = 12;
  p->coarse_iters = 3;
  p->coarse_size = 0;
  p->max_levels = 64;
  p->drop_R = 0.01;
  p->drop_Ac = 0.001;
  p->n_smooth_up = 2;
  p->precision = AIRG_FP64;
  p->keep_setup = 0;
  p->seed = 240808262ULL;
  p->sparsity_order = 1;
  p->matrix_free = 0;
  p->ideal_prolong = 0;
}

static int setup_common(const airg_csr* A, const airg_params* p, airg_stream_t stream, airg_hierarchy** out,
                        const airg_hierarchy* T, int reuse_levels, bool host_input = false) {
  if (!out) return AIRG_ERR_ARG;
  *out = nullptr;
  AIRG_TRY(check_csr_arg(A));
  AIRG_TRY(check_params(p));
  if (A->n == 0) return AIRG_ERR_ARG;
  if (T && T->n0 != A->n) return AIRG_ERR_ARG;
  airg_hierarchy* H = new (std::nothrow) airg_hierarchy;
  if (!H) return AIRG_ERR_OOM;
  H->p = *p;
  H->s = (cudaStream_t)stream;
  {
    const char* g = getenv("AIRG_NO_GRAPH");
    H->use_graph = (g && g[0] == '1') ? 0 : 1;
  }
  H->solve_mem.s = H->s;
  H->setup_mem.s = H->s;
  {
    // keep freed stream-ordered allocations cached in the pool between setup phases
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ULL;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
  }
  auto t0 = std::chrono::steady_clock::now();
  int rc = setup_impl(H, A, T, reuse_levels, host_input);
  if (rc != AIRG_OK) {
    cudaGetLastError();
    destroy(H);
    return rc;
  }
  H->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = H;
  return AIRG_OK;
}

int airg_setup(const airg_csr* A, const airg_params* p, airg_stream_t stream, airg_hierarchy** out) {
  return setup_common(A, p, stream, out, nullptr, 0);
}

int airg_setup_host(const airg_csr* A_host, const airg_params* p, airg_stream_t stream, airg_hierarchy** out) {
  return setup_common(A_host, p, stream, out, nullptr, 0, true);
}

int airg_setup_many(const airg_csr* As, int nsys, const airg_params* p, int nthreads, airg_stream_t stream,
                    airg_hierarchy** outs) {
  if (!As || !outs || nsys <= 0) return AIRG_ERR_ARG;
  for (int q = 0; q < nsys; ++q) outs[q] = nullptr;
  AIRG_TRY(check_params(p));
  for (int q = 0; q < nsys; ++q) AIRG_TRY(check_csr_arg(&As[q]));
  int dev = 0;
  CU_TRY(cudaGetDevice(&dev));
  // the inputs may still be being written on the caller's stream
  CU_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  const int nt = std::max(1, std::min(nthreads <= 0 ? 8 : nthreads, nsys));
  std::atomic<int> next{0};
  std::vector<int> rcs(nsys, AIRG_OK);
  auto work = [&]() {
    cudaSetDevice(dev);
    cudaStream_t ws = nullptr;
    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (int q; (q = next.fetch_add(1)) < nsys;) rcs[q] = AIRG_ERR_CUDA;
      return;
    }
    for (int q; (q = next.fetch_add(1)) < nsys;) {
      rcs[q] = setup_common(&As[q], p, (airg_stream_t)ws, &outs[q], nullptr, 0);
      if (rcs[q] == AIRG_OK && cudaStreamSynchronize(ws) != cudaSuccess) rcs[q] = AIRG_ERR_CUDA;
    }
    cudaStreamSynchronize(ws);
    cudaStreamDestroy(ws);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  int rc = AIRG_OK;
  for (int q = 0; q < nsys; ++q)
    if (rcs[q] != AIRG_OK && rc == AIRG_OK) rc = rcs[q];
  if (rc != AIRG_OK) {
    for (int q = 0; q < nsys; ++q) {
      if (outs[q]) outs[q]->s = (cudaStream_t)stream;
      airg_free(outs[q]);
      outs[q] = nullptr;
    }
    return rc;
  }
  // every hierarchy now belongs to the caller's stream (the worker streams are gone)
  for (int q = 0; q < nsys; ++q) {
    airg_hierarchy* H = outs[q];
    H->s = (cudaStream_t)stream;
    H->solve_mem.s = H->s;
    H->setup_mem.s = H->s;
  }
  return AIRG_OK;
}

int airg_setup_reuse(const airg_csr* A, const airg_params* p, const airg_hierarchy* T, int levels,
                     airg_stream_t stream, airg_hierarchy** out) {
  if (!T) {
    if (out) *out = nullptr;
    return AIRG_ERR_ARG;
  }
  return setup_common(A, p, stream, out, T, levels);
}

int airg_solve(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* opts, airg_solve_info* info,
               airg_stream_t stream) {
  if (!H || !b || !x || !opts) return AIRG_ERR_ARG;
  if (opts->restart < 1 || opts->restart > 32 || opts->max_it < 0 || !(opts->rtol >= 0.0)) return AIRG_ERR_ARG;
  airg_solve_info local{};
  airg_solve_info* inf = info ? info : &local;
  H->s = (cudaStream_t)stream;
  H->solve_mem.s = H->s;
  inf->levels = (int)H->lv.size();
  int rc;
  if (opts->outer == AIRG_OUTER_RICHARDSON) rc = solve_richardson(H, b, x, opts, inf);
  else if (opts->outer == AIRG_OUTER_FGMRES) rc = solve_fgmres(H, b, x, opts, inf);
  else return AIRG_ERR_ARG;
  inf->status = rc;
  return rc;
}

int airg_solve_host(airg_hierarchy* H, const double* b_host, double* x_host, const airg_solve_opts* opts,
                    airg_solve_info* info, airg_stream_t stream) {
  if (!H || !b_host || !x_host || !opts) return AIRG_ERR_ARG;
  H->s = (cudaStream_t)stream;
  H->solve_mem.s = H->s;
  if (!H->hb) {
    AIRG_TRY(H->solve_mem.alloc(&H->hb, std::max(H->n0, 1)));
    AIRG_TRY(H->solve_mem.alloc(&H->hx, std::max(H->n0, 1)));
  }
  const size_t bytes = sizeof(double) * (size_t)H->n0;
  CU_TRY(cudaMemcpyAsync(H->hb, b_host, bytes, cudaMemcpyHostToDevice, H->s));
  if (!opts->x0_zero) CU_TRY(cudaMemcpyAsync(H->hx, x_host, bytes, cudaMemcpyHostToDevice, H->s));
  int rc = airg_solve(H, H->hb, H->hx, opts, info, stream);
  if (rc < 0) return rc;
  CU_TRY(cudaMemcpyAsync(x_host, H->hx, bytes, cudaMemcpyDeviceToHost, H->s));
  CU_TRY(cudaStreamSynchronize(H->s));
  return rc;
}

int airg_vcycle(airg_hierarchy* H, const double* b, double* x, airg_stream_t stream) {
  if (!H || !b || !x) return AIRG_ERR_ARG;
  H->s = (cudaStream_t)stream;
  H->solve_mem.s = H->s;
  AIRG_TRY(solve_alloc(H, 1));
  if (H->pos0) dev_permute(b, H->pos0, H->bp, H->n0, false, H->s);
  else CU_TRY(cudaMemcpyAsync(H->bp, b, sizeof(double) * H->n0, cudaMemcpyDeviceToDevice, H->s));
  AIRG_TRY(vcycle_apply(H, H->bp, H->xp));
  if (H->pos0) dev_permute(H->xp, H->pos0, x, H->n0, true, H->s);
  else CU_TRY(cudaMemcpyAsync(x, H->xp, sizeof(double) * H->n0, cudaMemcpyDeviceToDevice, H->s));
  CU_TRY(cudaGetLastError());
  CU_TRY(cudaStreamSynchronize(H->s));
  AIRG_TRY(prof_flush(H));
  return AIRG_OK;
}

int airg_cf_split(const airg_csr* A, const airg_params* p, int level, int8_t* cf_out, airg_stream_t stream) {
  AIRG_TRY(check_csr_arg(A));
  AIRG_TRY(check_params(p));
  if (!cf_out || level < 0) return AIRG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp;
  tmp.s = s;
  DCsr D;
  D.nrows = D.ncols = A->n;
  D.nnz = A->nnz;
  D.rp = const_cast<int*>(A->rowptr);
  D.ci = const_cast<int*>(A->col);
  D.v = const_cast<double*>(A->val);
  int rc = validate_csr(D, tmp, s);
  int nf = 0;
  if (rc == AIRG_OK) rc = cf_split(D, to_setup(*p), level, cf_out, nullptr, &nf, tmp, s);
  if (rc == AIRG_OK) rc = cuda_status(cudaStreamSynchronize(s));
  tmp.release();
  cudaStreamSynchronize(s);
  return rc;
}

int airg_ddc_theta(const airg_csr* A, const int8_t* cf, double* theta, airg_stream_t stream) {
  AIRG_TRY(check_csr_arg(A));
  if (!cf || !theta) return AIRG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Arena tmp;
  tmp.s = s;
  DCsr D;
  D.nrows = D.ncols = A->n;
  D.nnz = A->nnz;
  D.rp = const_cast<int*>(A->rowptr);
  D.ci = const_cast<int*>(A->col);
  D.v = const_cast<double*>(A->val);
  int rc = validate_csr(D, tmp, s);
  if (rc == AIRG_OK) rc = ddc_theta(D, cf, theta, tmp, s);
  if (rc == AIRG_OK) rc = cuda_status(cudaStreamSynchronize(s));
  tmp.release();
  cudaStreamSynchronize(s);
  return rc;
}

void airg_free(airg_hierarchy* H) { destroy(H); }

int airg_num_levels(const airg_hierarchy* H) { return H ? (int)H->lv.size() : AIRG_ERR_ARG; }

int airg_level_info(const airg_hierarchy* H, int level, int64_t* info) {
  if (!H || !info) return AIRG_ERR_ARG;
  for (int i = 0; i < 16; ++i) info[i] = 0;
  if (level == -1) {
    info[0] = (int64_t)H->lv.size();
    info[1] = (int64_t)std::llround(H->grid_cx * 1e6);
    info[2] = (int64_t)std::llround(H->op_cx * 1e6);
    info[3] = (int64_t)std::llround(H->storage_cx * 1e6);
    info[4] = (int64_t)std::llround(H->setup_ms * 1e3);
    double tot[5] = {0, 0, 0, 0, 0};
    for (auto& v : H->phase_ms)
      for (int k = 0; k < 5; ++k) tot[k] += v[k];
    for (int k = 0; k < 5; ++k) info[5 + k] = (int64_t)std::llround(tot[k] * 1e3);
    info[10] = (int64_t)std::llround(H->layout_ms * 1e3);
    info[11] = H->A0s.sell ? 1 : 0;
    return AIRG_OK;
  }
  if (level < 0 || level >= (int)H->lb.size()) return AIRG_ERR_ARG;
  const LevelBuild& L = H->lb[level];
  const SolveLevel& S = H->lv[level];
  info[0] = L.n;
  info[1] = L.A.nnz;
  info[2] = L.nf;
  info[3] = L.nc;
  info[4] = L.Aff.nnz;
  info[5] = L.Afc.nnz;
  info[6] = L.Ainv.nnz;
  info[7] = L.Z.nnz;
  info[8] = L.coarsest ? 1 : 0;
  info[9] = L.Acf.nnz;
  info[10] = L.fitted;
  info[11] = S.AF.nnz;
  info[16] = L.W.nnz;
  info[17] = (S.AF.sell ? 1 : 0) | (S.Ainv.sell ? 2 : 0) | (S.Z.sell ? 4 : 0) | (S.A.sell ? 8 : 0) |
             (S.Aff.sell ? 16 : 0) | (S.W.sell ? 32 : 0);
  if (level < (int)H->phase_ms.size())
  {
    const auto& ph = H->phase_ms[level];
    info[12] = (int64_t)std::llround((ph[0] + ph[1]) * 1e3);  // CF splitting + extraction
    info[13] = (int64_t)std::llround(ph[2] * 1e3);            // polynomial fit and assembly
    info[14] = (int64_t)std::llround(ph[3] * 1e3);            // restrictor product
    info[15] = (int64_t)std::llround(ph[4] * 1e3);            // prolongator and coarse matrix
  }
  return AIRG_OK;
}

int airg_export_csr(const airg_hierarchy* H, int level, int which, int32_t* rowptr, int32_t* col, double* val) {
  if (!H || level < 0 || level >= (int)H->lb.size()) return AIRG_ERR_ARG;
  if ((which < 7 || which == 12) && !H->kept) return AIRG_ERR_ARG;
  const LevelBuild& L = H->lb[level];
  const SolveLevel& S = H->lv[level];
  const DCsr* M = nullptr;
  switch (which) {
    case 7: M = &S.AF; break;
    case 8: M = &S.Z; break;
    case 9: M = &H->A0s; break;
    case 10: M = &S.Ainv; break;
    case 11: M = &S.A; break;
    case 12: M = &L.W; break;
    case 13: M = &S.W; break;
    case 0: M = &L.A; break;
    case 1: M = &L.Aff; break;
    case 2: M = &L.Afc; break;
    case 3: M = &L.Acf; break;
    case 5: M = &L.Ainv; break;
    case 6: M = &L.Z; break;
    default: return AIRG_ERR_ARG;
  }
  if (L.coarsest && which != 0 && which != 5 && which != 9 && which != 10 && which != 11) return AIRG_ERR_ARG;
  if ((which == 12 || which == 13) && M->nrows == 0) return AIRG_ERR_ARG;  // one-point level: no W
  if (!L.coarsest && which == 11) return AIRG_ERR_ARG;
  cudaStream_t s = H->s;
  if (rowptr) CU_TRY(cudaMemcpyAsync(rowptr, M->rp, sizeof(int) * ((size_t)M->nrows + 1), cudaMemcpyDeviceToHost, s));
  if (col && M->nnz) CU_TRY(cudaMemcpyAsync(col, M->ci, sizeof(int) * (size_t)M->nnz, cudaMemcpyDeviceToHost, s));
  if (val && M->nnz) CU_TRY(cudaMemcpyAsync(val, M->v, sizeof(double) * (size_t)M->nnz, cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaStreamSynchronize(s));
  return AIRG_OK;
}

int airg_export_vectors(const airg_hierarchy* H, int level, int8_t* cf, int32_t* w, double* alpha) {
  if (!H || level < 0 || level >= (int)H->lb.size()) return AIRG_ERR_ARG;
  const LevelBuild& L = H->lb[level];
  cudaStream_t s = H->s;
  if ((cf || w) && !H->kept) return AIRG_ERR_ARG;
  if (cf && !L.coarsest) CU_TRY(cudaMemcpyAsync(cf, L.cf, (size_t)L.n, cudaMemcpyDeviceToHost, s));
  if (w && !L.coarsest && L.nf) CU_TRY(cudaMemcpyAsync(w, L.w, sizeof(int) * (size_t)L.nf, cudaMemcpyDeviceToHost, s));
  if (alpha)
    for (size_t k = 0; k < H->alphas[level].size(); ++k) alpha[k] = H->alphas[level][k];
  CU_TRY(cudaStreamSynchronize(s));
  return AIRG_OK;
}

int airg_export_layout(const airg_hierarchy* H, int level, int32_t* pos, int32_t* w_solve) {
  if (!H || level < 0 || level >= (int)H->lv.size()) return AIRG_ERR_ARG;
  const SolveLevel& S = H->lv[level];
  cudaStream_t s = H->s;
  if (pos) {
    if (!S.coarsest && S.lay) CU_TRY(cudaMemcpyAsync(pos, S.lay, sizeof(int) * (size_t)S.n, cudaMemcpyDeviceToHost, s));
    else
      for (int i = 0; i < S.n; ++i) pos[i] = i;
  }
  if (w_solve && !S.coarsest && S.nf)
    CU_TRY(cudaMemcpyAsync(w_solve, S.w, sizeof(int) * (size_t)S.nf, cudaMemcpyDeviceToHost, s));
  CU_TRY(cudaStreamSynchronize(s));
  return AIRG_OK;
}

int airg_profile_enable(airg_hierarchy* H, int enable) {
  if (!H) return AIRG_ERR_ARG;
  if (enable && !H->bytes_A0) {
    const double vb = H->vt == 0 ? 8.0 : (H->vt == 1 ? 4.0 : 2.0), xb = H->vt == 0 ? 8.0 : 4.0;
    for (auto& S : H->lv) {
      if (S.coarsest) S.bytes_A = spmv_bytes(S.A, true, vb, xb);
      S.bytes_Ainv = spmv_bytes(S.Ainv, true, vb, xb);
      if (!S.coarsest) {
        S.bytes_AF = spmv_bytes(S.AF, true, vb, xb);
        S.bytes_Z = spmv_bytes(S.Z, true, vb, xb);
        if (S.W.nrows > 0) S.bytes_W = spmv_bytes(S.W, false, vb, xb);
      }
      if (H->p.matrix_free) {
        // m - 1 SpMVs that read r in their epilogue, y = alpha r, and x += y
        const DCsr& M = S.coarsest ? S.A : S.Aff;
        const double n = M.nrows;
        S.bytes_mf = S.m > 1 ? (S.m - 1) * spmv_bytes(M, true) + 16.0 * n + 24.0 * n : 24.0 * n;
      }
    }
    H->bytes_A0 = spmv_bytes(H->A0s, false);
    H->bytes_V = vcycle_bytes(H);
  }
  H->prof.on = enable != 0;
  H->prof.mask = (unsigned)enable;
  for (int c = 0; c < PC_N; ++c) {
    H->prof.launches[c] = 0;
    H->prof.ms[c] = 0.0;
    H->prof.bytes[c] = 0.0;
    for (int l = 0; l < Profiler::kMaxLv; ++l) {
      H->prof.lv_launches[l][c] = 0;
      H->prof.lv_ms[l][c] = 0.0;
      H->prof.lv_bytes[l][c] = 0.0;
    }
  }
  return AIRG_OK;
}

int airg_kernel_times(airg_hierarchy* H, int64_t* launches, double* ms, double* bytes, int nclasses) {
  if (!H || nclasses < 0) return AIRG_ERR_ARG;
  AIRG_TRY(prof_flush(H));
  for (int c = 0; c < nclasses && c < PC_N; ++c) {
    if (launches) launches[c] = H->prof.launches[c];
    if (ms) ms[c] = H->prof.ms[c];
    if (bytes) bytes[c] = H->prof.bytes[c];
  }
  return AIRG_OK;
}

int64_t airg_launch_count(void) { return (int64_t)g_launches.load(); }

int airg_kernel_times_level(airg_hierarchy* H, int level, int64_t* launches, double* ms, double* bytes, int nclasses) {
  if (!H || nclasses < 0 || level < 0 || level >= Profiler::kMaxLv) return AIRG_ERR_ARG;
  AIRG_TRY(prof_flush(H));
  for (int c = 0; c < nclasses && c < PC_N; ++c) {
    if (launches) launches[c] = H->prof.lv_launches[level][c];
    if (ms) ms[c] = H->prof.lv_ms[level][c];
    if (bytes) bytes[c] = H->prof.lv_bytes[level][c];
  }
  return AIRG_OK;
}

const char* airg_status_string(int status) {
  switch (status) {
    case AIRG_OK: return "ok";
    case AIRG_NOT_CONVERGED: return "not converged (max_it reached)";
    case AIRG_ERR_ARG: return "invalid argument";
    case AIRG_ERR_CSR: return "invalid CSR (row pointers, column range, order or duplicates)";
    case AIRG_ERR_ZERO_DIAG: return "missing or zero diagonal entry";
    case AIRG_ERR_NAN: return "NaN or Inf in the solve";
    case AIRG_ERR_OOM: return "device out of memory";
    case AIRG_ERR_CUDA: return "CUDA runtime error";
    case AIRG_ERR_UNSUPPORTED: return "product row exceeds the working-set limit";
    case AIRG_ERR_SCRATCH: return "input exceeds the fixed scratch array of airg_cf_split_noalloc";
    default: return "unknown status";
  }
}

}  // extern "C"
