// Solve phase: the AIRG V-cycle (Section "Results": restriction with R = [Z I], recursion,
// one-point prolongation, up F-point smoothing only; coarsest level: iterations of the assembled
// GMRES polynomial) and the outer iterations (right-preconditioned FGMRES with CGS2, or the
// paper's undamped Richardson).  All vectors are kept in the level-0 F-then-C numbering; the
// permutation is applied once on entry and once on exit.
#include <cmath>
#include <cstring>

#include "airg_hier.cuh"

namespace airg {

// ------------------------------------------------------------------------------------------
// Kernel timing (only when profiling is enabled)
// ------------------------------------------------------------------------------------------
static cudaEvent_t prof_event(Profiler& P) {
  std::vector<cudaEvent_t>& pool = P.capturing ? P.graph_pool : P.pool;
  size_t& used = P.capturing ? P.graph_used : P.used;
  if (used == pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
  }
  return pool[used++];
}
struct ProfScope {
  Profiler& P;
  cudaStream_t s;
  int cls;
  double bytes;
  int level;
  cudaEvent_t a = nullptr;
  ProfScope(Profiler& P_, cudaStream_t s_, int c, double b, int lv = 0) : P(P_), s(s_), cls(c), bytes(b), level(lv) {
    if (P.on && ((P.mask >> cls) & 1u)) {
      a = prof_event(P);
      // inside a stream capture the record must become an event node of the graph
      if (a) cudaEventRecordWithFlags(a, s, P.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(P);
      if (b) {
        cudaEventRecordWithFlags(b, s, P.capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        (P.capturing ? P.graph_recs : P.pending).push_back({cls, level, a, b, bytes});
      }
    }
  }
};

static void prof_add(Profiler& P, const Profiler::Rec& r) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
    P.launches[r.cls] += 1;
    P.ms[r.cls] += ms;
    P.bytes[r.cls] += r.bytes;
    const int lv = std::min(r.level, Profiler::kMaxLv - 1);
    P.lv_launches[lv][r.cls] += 1;
    P.lv_ms[lv][r.cls] += ms;
    P.lv_bytes[lv][r.cls] += r.bytes;
  }
  cudaGetLastError();
}

// Reads the events of the last graph replay (the caller has synchronised the stream).
int prof_graph_read(airg_hierarchy* H) {
  Profiler& P = H->prof;
  if (P.graph_unread > 0) {
    for (auto& r : P.graph_recs) prof_add(P, r);
    P.graph_unread = 0;
  }
  return AIRG_OK;
}

int prof_flush(airg_hierarchy* H) {
  Profiler& P = H->prof;
  if (P.graph_unread > 0) {
    CU_TRY(cudaStreamSynchronize(H->s));
    prof_graph_read(H);
  }
  if (P.pending.empty()) return AIRG_OK;
  CU_TRY(cudaStreamSynchronize(H->s));
  for (auto& r : P.pending) prof_add(P, r);
  P.pending.clear();
  P.used = 0;
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Workspaces
// ------------------------------------------------------------------------------------------
int solve_alloc(airg_hierarchy* H, int restart) {
  if (H->restart_alloc >= restart && H->V) return AIRG_OK;
  Arena& a = H->solve_mem;
  const size_t n = (size_t)std::max(H->n0, 1);
  AIRG_TRY(a.alloc(&H->V, n * (restart + 1)));
  AIRG_TRY(a.alloc(&H->Zk, n * restart));
  if (!H->w) {
    AIRG_TRY(a.alloc(&H->w, n));
    AIRG_TRY(a.alloc(&H->r, n));
    AIRG_TRY(a.alloc(&H->bwork, n));
    AIRG_TRY(a.alloc(&H->rtmp, n));
    if (H->p.matrix_free) {
      AIRG_TRY(a.alloc(&H->mf_y, n));
      AIRG_TRY(a.alloc(&H->mf_y2, n));
    }
    AIRG_TRY(a.alloc(&H->bp, n));
    AIRG_TRY(a.alloc(&H->xp, n));
    AIRG_TRY(a.alloc(&H->dsc, 256));
    AIRG_TRY(reducer_init(H->red, a, H->s));
    if (!H->hsc) CU_TRY(cudaMallocHost((void**)&H->hsc, 256 * sizeof(double)));
  }
  H->restart_alloc = restart;
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// V-cycle.  b0: level-0 rhs (solve numbering, not modified); x0: output (n0 entries).  Level l's
// rhs lives in bwork[off_l, off_l + n_l) for l >= 1; level l's solution in x0[off_l, ...).
// ------------------------------------------------------------------------------------------
// Matrix-free polynomial (Section "AIRG": the stationary polynomial applied without assembling
// it): x = q(A) r, or x += q(A) r with `accumulate`, where q(A) = sum_{k<m} alpha_k A^k, by Horner's
// rule: y = alpha_{m-1} r, then y = alpha_k r + A y for k = m-2 .. 0 (m - 1 products by A, each
// one SpMV with the alpha_k r term in its epilogue).  alpha: device, m entries.
static int poly_apply_mf(airg_hierarchy* H, const DCsr& A, int lanes, const double* alpha, int m, const double* r,
                         double* x, bool accumulate, cudaStream_t s) {
  const int n = A.nrows;
  if (m <= 0) {
    if (!accumulate) dev_fill(x, 0.0, n, s);
    return AIRG_OK;
  }
  if (m == 1) {
    dev_coef_axpy(alpha, r, x, n, accumulate, s);
    return AIRG_OK;
  }
  double* buf[2] = {H->mf_y, H->mf_y2};
  int cur = 0;
  dev_coef_axpy(alpha + (m - 1), r, buf[cur], n, false, s);
  for (int k = m - 2; k >= 0; --k) {
    double* out = (k == 0 && !accumulate) ? x : buf[cur ^ 1];
    AIRG_TRY(dev_spmv_axpb(A, buf[cur], r, alpha + k, out, lanes, s));
    cur ^= 1;
  }
  if (accumulate) dev_add(buf[cur], x, n, s);
  return AIRG_OK;
}

double vcycle_bytes(const airg_hierarchy* H) {
  const int L = (int)H->lv.size() - 1;
  const bool mf = H->p.matrix_free != 0;
  double b = 0.0;
  for (int l = 0; l < L; ++l) {
    const SolveLevel& S = H->lv[l];
    const bool ideal = S.W.nrows > 0;
    b += S.bytes_Z;
    if (ideal) b += S.bytes_W;
    else if (H->p.n_smooth_up == 0) b += (double)S.nf * 16.0;
    for (int sm = 0; sm < H->p.n_smooth_up; ++sm)
      b += S.bytes_AF + (sm == 0 && !ideal ? 12.0 * S.nf : 0.0) + (mf ? S.bytes_mf : S.bytes_Ainv);
  }
  const SolveLevel& S = H->lv[L];
  const double inv = mf ? S.bytes_mf : S.bytes_Ainv;
  b += inv + (double)(H->p.coarse_iters - 1) * (S.bytes_A + inv);
  return b;
}

int vcycle_solve_order(airg_hierarchy* H, const double* b0, double* x0) {
  cudaStream_t s = H->s;
  Profiler& P = H->prof;
  const int L = (int)H->lv.size() - 1;
  auto bptr = [&](int l) -> const double* { return l == 0 ? b0 : H->bwork + H->lv[l].off; };
  // restriction down the hierarchy: b_{l+1} = b_C + Z b_F
  for (int l = 0; l < L; ++l) {
    const SolveLevel& S = H->lv[l];
    const double* bl = bptr(l);
    double* bn = H->bwork + H->lv[l + 1].off;
    ProfScope ps(P, s, PC_RESTRICT, S.bytes_Z, l);
    AIRG_TRY(dev_spmv(S.Z, bl, bl + S.nf, bn, SPMV_ADDB, S.lanes_Z, s));
  }
  // coarsest level: x = Ainv b, then x += Ainv (b - A x)
  {
    const SolveLevel& S = H->lv[L];
    const double* bl = bptr(L);
    double* xl = x0 + S.off;
    const bool mf = H->p.matrix_free != 0;
    {
      ProfScope ps(P, s, PC_COARSEST, mf ? S.bytes_mf : S.bytes_Ainv, L);
      if (mf) AIRG_TRY(poly_apply_mf(H, S.A, S.lanes_A, S.alpha, S.m, bl, xl, false, s));
      else AIRG_TRY(dev_spmv(S.Ainv, bl, nullptr, xl, SPMV_SET, S.lanes_Ainv, s));
    }
    for (int it = 1; it < H->p.coarse_iters; ++it) {
      {
        ProfScope ps(P, s, PC_COARSEST, S.bytes_A, L);
        AIRG_TRY(dev_spmv(S.A, xl, bl, H->rtmp, SPMV_RESID, S.lanes_A, s));
      }
      ProfScope ps(P, s, PC_COARSEST, mf ? S.bytes_mf : S.bytes_Ainv, L);
      if (mf) AIRG_TRY(poly_apply_mf(H, S.A, S.lanes_A, S.alpha, S.m, H->rtmp, xl, true, s));
      else AIRG_TRY(dev_spmv(S.Ainv, H->rtmp, nullptr, xl, SPMV_ADD, S.lanes_Ainv, s));
    }
  }
  // prolongation and up F-point smoothing
  for (int l = L - 1; l >= 0; --l) {
    const SolveLevel& S = H->lv[l];
    const double* bl = bptr(l);
    double* xl = x0 + S.off;
    const bool ideal = S.W.nrows > 0;
    if (ideal) {  // x_F = W x_C (approximate ideal prolongator)
      ProfScope ps(P, s, PC_PROLONG, S.bytes_W, l);
      AIRG_TRY(dev_spmv(S.W, xl + S.nf, nullptr, xl, SPMV_SET, S.lanes_W, s));
    } else if (H->p.n_smooth_up == 0) {
      ProfScope ps(P, s, PC_PROLONG, (double)S.nf * 16.0, l);
      dev_gather_prolong(xl, S.nf, S.w, s);
    }
    for (int sm = 0; sm < H->p.n_smooth_up; ++sm) {
      {
        ProfScope ps(P, s, PC_SMOOTH_RESID, S.bytes_AF + (sm == 0 && !ideal ? 12.0 * S.nf : 0.0), l);
        if (sm == 0 && !ideal) AIRG_TRY(dev_spmv_resid_prolong(S.AF, xl, S.w, bl, H->rtmp, S.lanes_AF, s));
        else AIRG_TRY(dev_spmv(S.AF, xl, bl, H->rtmp, SPMV_RESID, S.lanes_AF, s));
      }
      if (H->p.matrix_free) {
        ProfScope ps(P, s, PC_SMOOTH_UPDATE, S.bytes_mf, l);
        AIRG_TRY(poly_apply_mf(H, S.Aff, S.lanes_Aff, S.alpha, S.m, H->rtmp, xl, true, s));
      } else {
        ProfScope ps(P, s, PC_SMOOTH_UPDATE, S.bytes_Ainv, l);
        AIRG_TRY(dev_spmv(S.Ainv, H->rtmp, nullptr, xl, SPMV_ADD, S.lanes_Ainv, s));
      }
    }
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

// The same V-cycle with float vectors and float/bf16 operator values (mixed-precision form).
static int vcycle_lo(airg_hierarchy* H, const float* b0, float* x0) {
  cudaStream_t s = H->s;
  Profiler& P = H->prof;
  const int L = (int)H->lv.size() - 1;
  const int vt = H->vt;
  auto bptr = [&](int l) -> const float* { return l == 0 ? b0 : H->bwork_f + H->lv[l].off; };
  for (int l = 0; l < L; ++l) {
    const SolveLevel& S = H->lv[l];
    const float* bl = bptr(l);
    float* bn = H->bwork_f + H->lv[l + 1].off;
    ProfScope ps(P, s, PC_RESTRICT, S.bytes_Z, l);
    AIRG_TRY(dev_spmv_lo(S.Z, S.lo_Z, vt, bl, bl + S.nf, bn, SPMV_ADDB, S.lanes_Z, nullptr, s));
  }
  {
    const SolveLevel& S = H->lv[L];
    const float* bl = bptr(L);
    float* xl = x0 + S.off;
    {
      ProfScope ps(P, s, PC_COARSEST, S.bytes_Ainv, L);
      AIRG_TRY(dev_spmv_lo(S.Ainv, S.lo_Ainv, vt, bl, nullptr, xl, SPMV_SET, S.lanes_Ainv, nullptr, s));
    }
    for (int it = 1; it < H->p.coarse_iters; ++it) {
      {
        ProfScope ps(P, s, PC_COARSEST, S.bytes_A, L);
        AIRG_TRY(dev_spmv_lo(S.A, S.lo_A, vt, xl, bl, H->rtmp_f, SPMV_RESID, S.lanes_A, nullptr, s));
      }
      ProfScope ps(P, s, PC_COARSEST, S.bytes_Ainv, L);
      AIRG_TRY(dev_spmv_lo(S.Ainv, S.lo_Ainv, vt, H->rtmp_f, nullptr, xl, SPMV_ADD, S.lanes_Ainv, nullptr, s));
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const SolveLevel& S = H->lv[l];
    const float* bl = bptr(l);
    float* xl = x0 + S.off;
    if (H->p.n_smooth_up == 0) dev_gather_prolong_f(xl, S.nf, S.w, s);
    for (int sm = 0; sm < H->p.n_smooth_up; ++sm) {
      {
        ProfScope ps(P, s, PC_SMOOTH_RESID, S.bytes_AF, l);
        AIRG_TRY(dev_spmv_lo(S.AF, S.lo_AF, vt, xl, bl, H->rtmp_f, SPMV_RESID, S.lanes_AF, sm == 0 ? S.w : nullptr, s));
      }
      ProfScope ps(P, s, PC_SMOOTH_UPDATE, S.bytes_Ainv, l);
      AIRG_TRY(dev_spmv_lo(S.Ainv, S.lo_Ainv, vt, H->rtmp_f, nullptr, xl, SPMV_ADD, S.lanes_Ainv, nullptr, s));
    }
  }
  KERNEL_CHECK();
  return AIRG_OK;
}

// V-cycle through a CUDA graph: captured once per hierarchy (and again if the timed kernel classes
// change) on an internal stream, replayed on the caller's stream between two device copies.
static int ensure_vgraph(airg_hierarchy* H) {
  Profiler& P = H->prof;
  const unsigned mask = P.on ? P.mask : 0u;
  if (H->vg_exec && H->vg_mask == mask) return AIRG_OK;
  if (H->vg_exec) {
    if (P.graph_unread) {
      CU_TRY(cudaStreamSynchronize(H->s));
      prof_graph_read(H);
    }
    cudaGraphExecDestroy(H->vg_exec);
    H->vg_exec = nullptr;
  }
  if (!H->gin) {
    AIRG_TRY(H->solve_mem.alloc(&H->gin, std::max(H->n0, 1)));
    AIRG_TRY(H->solve_mem.alloc(&H->gout, std::max(H->n0, 1)));
  }
  if (H->vt && !H->gin_f) {
    const size_t n = (size_t)std::max(H->n0, 1);
    AIRG_TRY(H->solve_mem.alloc(&H->gin_f, n));
    AIRG_TRY(H->solve_mem.alloc(&H->gout_f, n));
    AIRG_TRY(H->solve_mem.alloc(&H->bwork_f, n));
    AIRG_TRY(H->solve_mem.alloc(&H->rtmp_f, n));
  }
  if (!H->cap_stream) CU_TRY(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
  cudaStream_t saved = H->s;
  H->s = H->cap_stream;
  P.capturing = true;
  P.graph_recs.clear();
  P.graph_used = 0;
  const long long launches0 = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc = (e == cudaSuccess) ? (H->vt ? vcycle_lo(H, H->gin_f, H->gout_f) : vcycle_solve_order(H, H->gin, H->gout))
                               : cuda_status(e);
  // captured kernels run only when the graph is replayed: count them there
  H->vg_kernels = g_launches.load() - launches0;
  g_launches.fetch_sub(H->vg_kernels);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(H->cap_stream, &g) : cudaSuccess;
  H->s = saved;
  P.capturing = false;
  if (rc == AIRG_OK && e2 != cudaSuccess) rc = cuda_status(e2);
  if (rc == AIRG_OK) rc = cuda_status(cudaGraphInstantiate(&H->vg_exec, g, 0));
  if (g) cudaGraphDestroy(g);
  if (rc != AIRG_OK) {
    cudaGetLastError();
    H->vg_exec = nullptr;
    return rc;
  }
  H->vg_mask = mask;
  return AIRG_OK;
}

int vcycle_apply(airg_hierarchy* H, const double* b0, double* x0) {
  if (!H->use_graph && !H->vt) {
    ProfScope pv(H->prof, H->s, PC_VCYCLE, H->bytes_V);
    return vcycle_solve_order(H, b0, x0);
  }
  AIRG_TRY(ensure_vgraph(H));
  if (H->vt) {  // FP64 in, float V-cycle, FP64 out
    if (H->prof.graph_unread) {
      CU_TRY(cudaStreamSynchronize(H->s));
      prof_graph_read(H);
    }
    dev_cast_d2f(b0, H->gin_f, H->n0, H->s);
    {
      ProfScope pv(H->prof, H->s, PC_VCYCLE, H->bytes_V);
      CU_TRY(cudaGraphLaunch(H->vg_exec, H->s));
    }
    g_launches.fetch_add(H->vg_kernels);
    if (!H->prof.graph_recs.empty()) H->prof.graph_unread = 1;
    dev_cast_f2d(H->gout_f, x0, H->n0, H->s);
    KERNEL_CHECK();
    return AIRG_OK;
  }
  const size_t bytes = sizeof(double) * (size_t)H->n0;
  if (H->prof.graph_unread) {  // the previous replay's events have not been read yet
    CU_TRY(cudaStreamSynchronize(H->s));
    prof_graph_read(H);
  }
  CU_TRY(cudaMemcpyAsync(H->gin, b0, bytes, cudaMemcpyDeviceToDevice, H->s));
  {
    ProfScope pv(H->prof, H->s, PC_VCYCLE, H->bytes_V);
    CU_TRY(cudaGraphLaunch(H->vg_exec, H->s));
  }
  g_launches.fetch_add(H->vg_kernels);
  if (!H->prof.graph_recs.empty()) H->prof.graph_unread = 1;
  CU_TRY(cudaMemcpyAsync(x0, H->gout, bytes, cudaMemcpyDeviceToDevice, H->s));
  return AIRG_OK;
}

// ------------------------------------------------------------------------------------------
// Outer iterations
// ------------------------------------------------------------------------------------------
static int read_scalars(airg_hierarchy* H, int count) {
  CU_TRY(cudaMemcpyAsync(H->hsc, H->dsc, sizeof(double) * count, cudaMemcpyDeviceToHost, H->s));
  CU_TRY(cudaStreamSynchronize(H->s));
  prof_graph_read(H);
  return AIRG_OK;
}

enum { DS_H1 = 0, DS_H2 = 64, DS_NRM = 128, DS_AUX = 129, DS_Y = 160 };

// true residual r = bp - A xp and its squared norm into hsc[DS_NRM]
static int true_residual(airg_hierarchy* H) {
  const int n = H->n0;
  {
    ProfScope ps(H->prof, H->s, PC_TOP_OP, H->bytes_A0);
    AIRG_TRY(dev_spmv(H->A0s, H->xp, H->bp, H->r, SPMV_RESID, H->lanes_A0, H->s));
  }
  AIRG_TRY(dev_nrm2sq(H->r, n, H->dsc + DS_NRM, H->red, H->s));
  return read_scalars(H, DS_NRM + 1);
}

static void to_solve_order(airg_hierarchy* H, const double* in, double* out) {
  if (H->pos0) dev_permute(in, H->pos0, out, H->n0, false, H->s);
  else cudaMemcpyAsync(out, in, sizeof(double) * H->n0, cudaMemcpyDeviceToDevice, H->s);
}
static void from_solve_order(airg_hierarchy* H, const double* in, double* out) {
  if (H->pos0) dev_permute(in, H->pos0, out, H->n0, true, H->s);
  else cudaMemcpyAsync(out, in, sizeof(double) * H->n0, cudaMemcpyDeviceToDevice, H->s);
}

static int start(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* o, double* bnorm) {
  const int n = H->n0;
  to_solve_order(H, b, H->bp);
  if (o->x0_zero) CU_TRY(cudaMemsetAsync(H->xp, 0, sizeof(double) * n, H->s));
  else to_solve_order(H, x, H->xp);
  AIRG_TRY(dev_nrm2sq(H->bp, n, H->dsc + DS_AUX, H->red, H->s));
  AIRG_TRY(read_scalars(H, DS_AUX + 1));
  *bnorm = std::sqrt(H->hsc[DS_AUX]);
  return AIRG_OK;
}

int solve_fgmres(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* o, airg_solve_info* info) {
  const int n = H->n0, restart = o->restart;
  cudaStream_t s = H->s;
  AIRG_TRY(solve_alloc(H, restart));
  double bn = 0.0;
  AIRG_TRY(start(H, b, x, o, &bn));
  int iters = 0;
  double relres = 0.0;
  int status = AIRG_OK;
  if (bn == 0.0) {
    CU_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    info->iters = 0;
    info->relres = 0.0;
    info->status = AIRG_OK;
    return AIRG_OK;
  }
  AIRG_TRY(true_residual(H));
  double beta = std::sqrt(H->hsc[DS_NRM]);
  relres = beta / bn;
  std::vector<double> Hh((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), y(restart);
  while (true) {
    if (!(relres == relres) || std::isinf(relres)) { status = AIRG_ERR_NAN; break; }
    if (relres <= o->rtol) break;
    if (iters >= o->max_it) { status = AIRG_NOT_CONVERGED; break; }
    dev_scale(H->r, beta, H->V, n, s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < restart && iters < o->max_it; ++j) {
      double* vj = H->V + (size_t)j * n;
      double* zj = H->Zk + (size_t)j * n;
      AIRG_TRY(vcycle_apply(H, vj, zj));
      {
        ProfScope ps(H->prof, s, PC_TOP_OP, H->bytes_A0);
        AIRG_TRY(dev_spmv(H->A0s, zj, nullptr, H->w, SPMV_SET, H->lanes_A0, s));
      }
      {
        ProfScope ps(H->prof, s, PC_GS, 8.0 * n * (3.0 * (j + 1) + 5.0));
        AIRG_TRY(dev_gs_pass(H->V, n, j + 1, H->w, n, nullptr, H->dsc + DS_H1, nullptr, H->red, s));
        AIRG_TRY(dev_gs_pass(H->V, n, j + 1, H->w, n, H->dsc + DS_H1, H->dsc + DS_H2, nullptr, H->red, s));
        AIRG_TRY(dev_gs_pass(H->V, n, j + 1, H->w, n, H->dsc + DS_H2, nullptr, H->dsc + DS_NRM, H->red, s));
      }
      AIRG_TRY(read_scalars(H, DS_NRM + 1));
      double* h = &Hh[(size_t)j * (restart + 1)];
      for (int i = 0; i <= j; ++i) h[i] = H->hsc[DS_H1 + i] + H->hsc[DS_H2 + i];
      const double hj1 = std::sqrt(H->hsc[DS_NRM]);
      h[j + 1] = hj1;
      for (int i = 0; i < j; ++i) {
        const double t1 = h[i], t2 = h[i + 1];
        h[i] = cs[i] * t1 + sn[i] * t2;
        h[i + 1] = -sn[i] * t1 + cs[i] * t2;
      }
      const double d = std::hypot(h[j], h[j + 1]);
      double c_ = 1.0, s_ = 0.0;
      if (d != 0.0) { c_ = h[j] / d; s_ = h[j + 1] / d; }
      h[j] = c_ * h[j] + s_ * h[j + 1];
      h[j + 1] = 0.0;
      cs[j] = c_;
      sn[j] = s_;
      g[j + 1] = -s_ * g[j];
      g[j] = c_ * g[j];
      iters++;
      const double est = std::fabs(g[j + 1]) / bn;
      if (est <= o->rtol || hj1 == 0.0 || !(est == est)) { ++j; break; }
      dev_scale(H->w, hj1, H->V + (size_t)(j + 1) * n, n, s);
    }
    const int k = j;
    for (int i = k - 1; i >= 0; --i) {
      double t = g[i];
      for (int q = i + 1; q < k; ++q) t -= Hh[(size_t)q * (restart + 1) + i] * y[q];
      y[i] = t / Hh[(size_t)i * (restart + 1) + i];
    }
    CU_TRY(cudaMemcpyAsync(H->dsc + DS_Y, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
    AIRG_TRY(dev_multi_axpy(H->Zk, n, k, H->dsc + DS_Y, H->xp, n, s));
    AIRG_TRY(true_residual(H));
    beta = std::sqrt(H->hsc[DS_NRM]);
    relres = beta / bn;
  }
  from_solve_order(H, H->xp, x);
  KERNEL_CHECK();
  CU_TRY(cudaStreamSynchronize(s));
  AIRG_TRY(prof_flush(H));
  info->iters = iters;
  info->relres = relres;
  info->status = status;
  return status;
}

int solve_richardson(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* o, airg_solve_info* info) {
  const int n = H->n0;
  cudaStream_t s = H->s;
  AIRG_TRY(solve_alloc(H, 1));
  double bn = 0.0;
  AIRG_TRY(start(H, b, x, o, &bn));
  int iters = 0, status = AIRG_OK;
  double relres = 0.0;
  if (bn == 0.0) {
    CU_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    info->iters = 0;
    info->relres = 0.0;
    info->status = AIRG_OK;
    return AIRG_OK;
  }
  const double one = 1.0;
  CU_TRY(cudaMemcpyAsync(H->dsc + DS_Y, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  while (true) {
    AIRG_TRY(true_residual(H));
    relres = std::sqrt(H->hsc[DS_NRM]) / bn;
    if (!(relres == relres) || std::isinf(relres)) { status = AIRG_ERR_NAN; break; }
    if (relres <= o->rtol) break;
    if (iters >= o->max_it) { status = AIRG_NOT_CONVERGED; break; }
    AIRG_TRY(vcycle_apply(H, H->r, H->Zk));
    AIRG_TRY(dev_multi_axpy(H->Zk, n, 1, H->dsc + DS_Y, H->xp, n, s));
    iters++;
  }
  from_solve_order(H, H->xp, x);
  KERNEL_CHECK();
  CU_TRY(cudaStreamSynchronize(s));
  AIRG_TRY(prof_flush(H));
  info->iters = iters;
  info->relres = relres;
  info->status = status;
  return status;
}

}  // namespace airg
