// The hierarchy object behind the opaque airg_hierarchy handle.
#pragma once
#include <deque>
#include <vector>

#include "airg_common.cuh"

namespace airg {

// Solve-phase data of one level, in the level's F-then-C numbering.
struct SolveLevel {
  int n = 0, nf = 0, nc = 0;
  long long off = 0;  // offset of this level's vector in the nested work buffers
  bool coarsest = false;
  DCsr AF;    // [A_ff A_fc] rows of the F-points, columns in F-then-C numbering (n_f x n)
  DCsr Ainv;  // Ainv_ff (n_f x n_f); on the coarsest level the whole-matrix polynomial
  DCsr Z;     // restrictor rows in the next level's numbering (n_c x n_f)
  int* w = nullptr;  // one-point prolongation source per F-point (next level's numbering)
  int* lay = nullptr;  // natural index of this level -> nested solve position (non-coarsest)
  int8_t* cf = nullptr;  // the level's CF splitting (non-coarsest), kept for setup re-use
  DCsr A;     // coarsest level only: the level matrix
  int lanes_AF = 4, lanes_Ainv = 4, lanes_Z = 4, lanes_A = 4;
  // mixed precision: the same operators with float or bf16 values (nullptr in FP64 mode)
  void *lo_AF = nullptr, *lo_Ainv = nullptr, *lo_Z = nullptr, *lo_A = nullptr;
  double bytes_AF = 0, bytes_Ainv = 0, bytes_Z = 0, bytes_A = 0;  // algorithmic bytes per SpMV
  // matrix-free polynomial application: A_ff (non-coarsest levels, F numbering) and the m
  // coefficients on the device; the coarsest level applies its polynomial with A
  DCsr Aff;
  // approximate ideal prolongator (rows n_f, columns in the next level's numbering); empty for
  // the one-point operator w
  DCsr W;
  int lanes_W = 4;
  double bytes_W = 0;
  double* alpha = nullptr;
  int m = 0, lanes_Aff = 4;
  double bytes_mf = 0;  // algorithmic bytes of one matrix-free application
};

// Kernel classes timed by the profiler.  PC_VCYCLE times each whole V-cycle application (the graph
// replay, or the eager sequence) with one event pair outside it, so it adds nothing inside the
// cycle; its bytes are the sum of the algorithmic bytes of every SpMV of the cycle.
enum ProfClass { PC_SMOOTH_RESID = 0, PC_SMOOTH_UPDATE, PC_RESTRICT, PC_TOP_OP, PC_COARSEST, PC_PROLONG, PC_GS, PC_VCYCLE, PC_N };

struct Profiler {
  bool on = false;
  unsigned mask = 0;  // bit c: time class c
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    int cls, level;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Rec> pending;
  // events recorded inside the captured V-cycle graph: read after every replay
  bool capturing = false;
  std::vector<cudaEvent_t> graph_pool;
  size_t graph_used = 0;
  std::vector<Rec> graph_recs;
  int graph_unread = 0;
  long long launches[PC_N] = {};
  double ms[PC_N] = {};
  double bytes[PC_N] = {};
  static constexpr int kMaxLv = 128;  // per-level sums (levels beyond the last slot are folded in)
  long long lv_launches[kMaxLv][PC_N] = {};
  double lv_ms[kMaxLv][PC_N] = {};
  double lv_bytes[kMaxLv][PC_N] = {};
};

}  // namespace airg

struct airg_hierarchy {
  airg_params p{};
  cudaStream_t s = nullptr;
  airg::Arena solve_mem;  // solve-phase operators and workspaces
  airg::Arena setup_mem;  // natural-numbering setup operators (released unless keep_setup)
  std::vector<airg::LevelBuild> lb;
  std::vector<std::vector<double>> alphas;  // host copies of each level's coefficients
  std::vector<airg::SolveLevel> lv;
  int n0 = 0;
  airg::DCsr A0s;  // top-level matrix in level-0 F-then-C numbering
  std::deque<airg::DSell> sells;  // sliced ELL copies the solve operators point to (DCsr::sell)
  int* pos0 = nullptr;  // natural -> solve numbering (nullptr: identity)
  int lanes_A0 = 4;
  double bytes_A0 = 0;
  double bytes_V = 0;  // algorithmic bytes of every SpMV of one V-cycle (vcycle_bytes)
  // workspaces (allocated on first solve)
  int restart_alloc = 0;
  double *V = nullptr, *Zk = nullptr, *w = nullptr, *r = nullptr, *bwork = nullptr, *rtmp = nullptr,
         *bp = nullptr, *xp = nullptr, *dsc = nullptr, *hb = nullptr, *hx = nullptr;
  double *mf_y = nullptr, *mf_y2 = nullptr;  // Horner iterates of the matrix-free polynomial
  double* hsc = nullptr;  // pinned host mirror of dsc
  airg::Reducer red{};
  airg::Profiler prof;
  // V-cycle as a CUDA graph over fixed buffers gin -> gout, captured on first use
  int use_graph = 1;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t vg_exec = nullptr;
  unsigned vg_mask = 0xffffffffu;
  long long vg_kernels = 0;  // kernel nodes in the graph (counted at every replay)
  double *gin = nullptr, *gout = nullptr;
  // mixed precision V-cycle (precision AIRG_FP32 or AIRG_BF16_VALUES): float work vectors
  int vt = 0;  // 0 FP64, 1 float values, 2 bf16 values
  float *gin_f = nullptr, *gout_f = nullptr, *bwork_f = nullptr, *rtmp_f = nullptr;
  // info
  double setup_ms = 0, grid_cx = 0, op_cx = 0, storage_cx = 0, layout_ms = 0;
  std::vector<std::vector<float>> phase_ms;  // per level: CF split, extraction, polynomial, Z, P + RAP
  long long top_nnz = 0;
  bool kept = false;
};

namespace airg {
int solve_alloc(airg_hierarchy* H, int restart);
int vcycle_solve_order(airg_hierarchy* H, const double* b0, double* x0);
// x0 = M b0 in the solve numbering, through the captured graph when enabled
int vcycle_apply(airg_hierarchy* H, const double* b0, double* x0);
int prof_graph_read(airg_hierarchy* H);
int solve_fgmres(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* o, airg_solve_info* info);
int solve_richardson(airg_hierarchy* H, const double* b, double* x, const airg_solve_opts* o, airg_solve_info* info);
int prof_flush(airg_hierarchy* H);
// Algorithmic bytes of one V-cycle: the sum of the byte counts its SpMV classes are timed with.
double vcycle_bytes(const airg_hierarchy* H);
}  // namespace airg
