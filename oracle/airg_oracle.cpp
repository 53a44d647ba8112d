// AIRG oracle: plain, slow, FP64 CPU restatement of the reduction multigrid of
// Dargaville, Smedley-Stevenson, Smith & Pain, "Coarsening and parallelism with reduction
// multigrids for hyperbolic Boltzmann transport" (arXiv 2408.08262).
//
// TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline leg of the
// benchmark load this library.  The CUDA library never calls, links or includes it, and it shares
// no code, header, table or helper with the CUDA library.
//
// Every function follows the paper step by step, in its order and notation, with no blocking,
// fusion or reordering:
//   strength of connection ............ Section "CF splitting", eq. soc (absolute values)
//   PMISR .............................. Algorithm 1, with the loop cap of Section "Parallel results"
//   DDC ................................ Algorithm 2, with the constant-fraction rule
//   extraction, GMRES polynomial fit ... Section "AIRG", setup steps 2-6, eq. gmres_poly
//   fixed-sparsity powers .............. eq. fixed_sparsity (first-order sparsity)
//   Z, one-point P, R A P, drops ....... setup steps 9-11, eq. prolong, relative row-wise inf-norm
//   V-cycle ............................ Section "Results": up F-point smoothing only, no down smooth
//   coarse solve ....................... Section "Timing results": GMRES polynomial iterations
//   outer iteration .................... undamped Richardson (paper) or right-preconditioned FGMRES
// Readings of silent or garbled passages are documented next to the code that takes them.
//
// Where arithmetic order can change the last bit, this code fixes the order to the plain
// definition: sums run in ascending index order; products accumulated by std::fma.  Compiled with
// -ffp-contract=off so the compiler adds no fusion of its own.  Everything runs on one thread
// except, on request (oracle_set_threads), the rows of the SpMV, which are independent: any
// thread count gives bitwise the same results.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------------------
// Sparse matrix (CSR, sorted unique columns)
// ---------------------------------------------------------------------------------------------
struct Csr {
  int nrows = 0, ncols = 0;
  std::vector<int> rp{0}, ci;
  std::vector<double> v;
  int nnz() const { return (int)ci.size(); }
};

Csr make_csr(int nr, int nc, const int* rp, const int* ci, const double* v) {
  Csr A;
  A.nrows = nr;
  A.ncols = nc;
  A.rp.assign(rp, rp + nr + 1);
  int nz = rp[nr];
  A.ci.assign(ci, ci + nz);
  A.v.assign(v, v + nz);
  return A;
}

// Threads of the SpMV row loop (1 unless oracle_set_threads asks for more; only the all-cores CPU
// baseline does).  Rows are independent and each keeps its own summation order, so any thread
// count gives bitwise the same result.
int g_threads = 1;

// y = A x, each row summed in ascending column order.
void spmv(const Csr& A, const std::vector<double>& x, std::vector<double>& y) {
  y.assign(A.nrows, 0.0);
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int i = 0; i < A.nrows; ++i) {
    double s = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) s += A.v[k] * x[A.ci[k]];
    y[i] = s;
  }
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}
double nrm2(const std::vector<double>& a) { return std::sqrt(dot(a, a)); }

double entry(const Csr& A, int i, int j) {  // a_ij or 0
  auto b = A.ci.begin() + A.rp[i], e = A.ci.begin() + A.rp[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it != e && *it == j) return A.v[it - A.ci.begin()];
  return 0.0;
}
bool has_entry(const Csr& A, int i, int j) {
  auto b = A.ci.begin() + A.rp[i], e = A.ci.begin() + A.rp[i + 1];
  auto it = std::lower_bound(b, e, j);
  return it != e && *it == j;
}

// ---------------------------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  The c-th output
// of a SplitMix64 stream seeded with `key` is mix(key + (c+1) * golden-gamma).
// ---------------------------------------------------------------------------------------------
const uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// stream 0: PMISR tie-break weights; stream 1: Box-Muller right-hand side.
uint64_t stream_key(uint64_t seed, int level, int stream) {
  return mix64(seed + kGamma * (uint64_t)(1 + 2 * level + stream));
}
double unif01(uint64_t key, uint64_t c) {  // [0, 1), 53 random bits
  return (double)(mix64(key + kGamma * (c + 1)) >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------------------------
// Parameters
// ---------------------------------------------------------------------------------------------
struct Params {
  double strong_threshold;
  double ddc_fraction;
  int pmisr_max_loops;
  int poly_order;  // degree d; m = d + 1 coefficients
  int coarse_poly_order;
  int coarse_iters;
  int coarse_size;
  int max_levels;
  double drop_R;
  double drop_Ac;
  int n_smooth_up;
  int one_point_weighted;  // 0: weight 1 (default); reserved
  uint64_t seed;
  int sparsity_order;      // 1: pattern(A_ff) (default); 2: pattern(A_ff^2)
  int matrix_free;         // 1: the V-cycle applies q(A_ff) (q(A) on the coarsest) from its definition
  int ideal_prolong;       // 1: approximate ideal prolongator W = -Ainv A_fc (eq. prolong) for P
};

// ---------------------------------------------------------------------------------------------
// CF splitting (Section "CF splitting")
// ---------------------------------------------------------------------------------------------
enum : int8_t { U = 0, F = 1, C = 2 };

// eq. soc: S_i = { j != i : |a_ij| >= alpha max_{k != i} |a_ik| }, absolute values (Section
// "Serial comparison").  Reading: stored zeros are never strong; a row with no nonzero
// off-diagonal has S_i empty.
std::vector<int8_t> strength(const Csr& A, double alpha) {
  std::vector<int8_t> s(A.nnz(), 0);
  for (int i = 0; i < A.nrows; ++i) {
    double mx = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] != i) mx = std::max(mx, std::fabs(A.v[k]));
    if (mx == 0.0) continue;
    double thr = alpha * mx;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      if (j == i || A.v[k] == 0.0) continue;
      if (std::fabs(A.v[k]) >= thr) s[k] = 1;
    }
  }
  return s;
}

struct Graph {  // symmetrised strong graph: S_i union S_i^T, as adjacency lists
  std::vector<std::vector<int>> nb;
  std::vector<int> nS, nST;  // |S_i|, |S_i^T|
};

Graph sym_graph(const Csr& A, const std::vector<int8_t>& s) {
  Graph g;
  int n = A.nrows;
  g.nb.assign(n, {});
  g.nS.assign(n, 0);
  g.nST.assign(n, 0);
  for (int i = 0; i < n; ++i)
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (s[k]) {
        int j = A.ci[k];
        g.nS[i]++;
        g.nST[j]++;
        g.nb[i].push_back(j);
        g.nb[j].push_back(i);
      }
  for (auto& v : g.nb) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  return g;
}

// Algorithm 1 (PMISR).  Readings:
//  * w_i = |S_i| + |S_i^T| + r_i with r_i in [0,1) from the seeded stream (counts are set sizes).
//  * the initial F set {w_i < 1} is therefore the set of nodes with no strong connection.
//  * the garbled loop guard is read as: at most max_loops rounds while unassigned nodes remain
//    (max_loops <= 0: no cap).
//  * D is formed from the state at the start of a round and compares only against *unassigned*
//    neighbours, with ties broken by index: (w_i, i) < (w_j, j).
//  * after the loop, unassigned nodes become C.
std::vector<int8_t> pmisr(const Graph& g, const std::vector<double>& w, int max_loops, int* rounds_out) {
  int n = (int)w.size();
  std::vector<int8_t> cf(n, U);
  for (int i = 0; i < n; ++i)
    if (w[i] < 1.0) cf[i] = F;
  int rounds = 0;
  for (int loop = 1;; ++loop) {
    if (max_loops > 0 && loop > max_loops) break;
    bool any_u = false;
    for (int i = 0; i < n; ++i) any_u |= (cf[i] == U);
    if (!any_u) break;
    std::vector<char> inD(n, 0);
    for (int i = 0; i < n; ++i) {
      if (cf[i] != U) continue;
      bool is_min = true;
      for (int j : g.nb[i]) {
        if (cf[j] != U) continue;
        if (!(w[i] < w[j] || (w[i] == w[j] && i < j))) { is_min = false; break; }
      }
      inD[i] = is_min;
    }
    for (int i = 0; i < n; ++i)
      if (inD[i]) {
        cf[i] = F;
        for (int k : g.nb[i])
          if (cf[k] == U) cf[k] = C;
      }
    rounds = loop;
  }
  for (int i = 0; i < n; ++i)
    if (cf[i] == U) cf[i] = C;
  if (rounds_out) *rounds_out = rounds;
  return cf;
}

// Row-wise diagonal dominance ratio of A_ff (Algorithm 2): theta_i = sum_{j in F, j != i} |a_ij|
// / |a_ii|, summed in ascending column order, for i in F (0 elsewhere).  A zero diagonal gives
// +inf (or 0 if the sum is 0).
std::vector<double> ddc_theta(const Csr& A, const std::vector<int8_t>& cf) {
  std::vector<double> th(A.nrows, 0.0);
  for (int i = 0; i < A.nrows; ++i) {
    if (cf[i] != F) continue;
    double s = 0.0, d = 0.0;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int j = A.ci[k];
      if (j == i) d = std::fabs(A.v[k]);
      else if (cf[j] == F) s += std::fabs(A.v[k]);
    }
    th[i] = (s == 0.0) ? 0.0 : s / d;
  }
  return th;
}

// Algorithm 2 (DDC) with alpha_diag chosen so that a constant fraction converts (the exact
// QuickSelect variant).  Readings: candidates are F-points with theta != 0 (Algorithm 2's
// "theta_i != 0"; diagonal rows are ignored); k = floor(fraction * |F|), capped by the number of
// candidates; tau = k-th largest candidate theta; every candidate with theta >= tau converts
// (ties may convert more than k).  theta is evaluated on the F set before any conversion.
std::vector<int8_t> ddc(const Csr& A, std::vector<int8_t> cf, double fraction, double* tau_out,
                        std::vector<double>* theta_out) {
  std::vector<double> th = ddc_theta(A, cf);
  if (theta_out) *theta_out = th;
  long nF = 0;
  std::vector<double> cand;
  for (int i = 0; i < A.nrows; ++i)
    if (cf[i] == F) {
      nF++;
      if (th[i] != 0.0) cand.push_back(th[i]);
    }
  long k = (long)std::floor(fraction * (double)nF);
  k = std::min<long>(k, (long)cand.size());
  double tau = INFINITY;
  if (k > 0) {
    std::sort(cand.begin(), cand.end(), [](double a, double b) { return a > b; });
    tau = cand[k - 1];
    for (int i = 0; i < A.nrows; ++i)
      if (cf[i] == F && th[i] != 0.0 && th[i] >= tau) cf[i] = C;
  }
  if (tau_out) *tau_out = tau;
  return cf;
}

struct CfDetail {
  std::vector<int8_t> strong, cf_pmisr, cf;
  std::vector<double> w, theta;
  double tau = INFINITY;
  int rounds = 0;
};

CfDetail cf_split(const Csr& A, const Params& p, int level) {
  CfDetail d;
  d.strong = strength(A, p.strong_threshold);
  Graph g = sym_graph(A, d.strong);
  int n = A.nrows;
  d.w.resize(n);
  uint64_t key = stream_key(p.seed, level, 0);
  for (int i = 0; i < n; ++i) d.w[i] = (double)(g.nS[i] + g.nST[i]) + unif01(key, (uint64_t)i);
  d.cf_pmisr = pmisr(g, d.w, p.pmisr_max_loops, &d.rounds);
  d.cf = ddc(A, d.cf_pmisr, p.ddc_fraction, &d.tau, &d.theta);
  return d;
}

// ---------------------------------------------------------------------------------------------
// GMRES polynomial (Section "AIRG", setup steps 3-8)
// ---------------------------------------------------------------------------------------------

// Step 3: normally distributed rhs (zero mean) by the Box-Muller transform in single precision:
// for entry i, k1 and k2 are the top 24 bits of outputs 2i and 2i+1 of stream 1,
// u1 = 1 - k1 2^-24 (in (0, 1]), u2 = k2 2^-24, z = sqrt(-2 ln u1) cos(2 pi u2).  ln and cos are
// evaluated by the fixed float sequences below, so that every implementation following them
// draws the same vector bit for bit; the paper asks only for a normally distributed rhs.
uint32_t unif24(uint64_t key, uint64_t c) { return (uint32_t)(mix64(key + kGamma * (c + 1)) >> 40); }

// ln x, x in (0, 1] normal: x = m 2^e with m in [1, 2), halved (e + 1) above sqrt 2; with f = m - 1
// and s = f / (2 + f), ln(1 + f) = 2 atanh s = 2 (s + s^3/3 + s^5/5 + ...) (Abramowitz & Stegun
// 4.1.28), here to s^11, by Horner in z = s^2; e ln 2 is added with ln 2 split in a short high
// part (exact products e * hi) and a low part.
float ln_f32(float x) {
  uint32_t bits;
  std::memcpy(&bits, &x, 4);
  int e = (int)(bits >> 23) - 127;
  uint32_t mbits = (bits & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &mbits, 4);
  if (m > 0x1.6a09e6p+0f) {  // sqrt 2
    m = m * 0.5f;
    e += 1;
  }
  const float f = m - 1.0f;
  const float s = f / (2.0f + f);
  const float z = s * s;
  float p = std::fmaf(z, 0x1.745d18p-3f, 0x1.c71c72p-3f);  // 2/11, 2/9
  p = std::fmaf(z, p, 0x1.24924ap-2f);                     // 2/7
  p = std::fmaf(z, p, 0x1.99999ap-2f);                     // 2/5
  p = std::fmaf(z, p, 0x1.555556p-1f);                     // 2/3
  const float sz = s * z;
  const float r = std::fmaf(sz, p, 2.0f * s);
  const float ef = (float)e;
  return std::fmaf(ef, 0x1.62e4p-1f, std::fmaf(ef, 0x1.7f7d1cp-20f, r));  // ln 2 = hi + lo
}

// cos(2 pi k 2^-24), k < 2^24: the nearest quarter turn q is removed exactly in integers, leaving
// x = 2 pi r with |r| <= 1/8; cos x and sin x by their Taylor series (to x^10 and x^9) by Horner in
// x^2, and cos(x + q pi/2) picked by q mod 4.
float cos2pi_f32(uint32_t k) {
  const uint32_t q = (k + (1u << 21)) >> 22;
  const int32_t ri = (int32_t)k - (int32_t)(q << 22);
  const float r = (float)ri * 0x1p-24f;
  const float x = r * 0x1.921fb6p+2f;  // 2 pi
  const float x2 = x * x;
  float c = std::fmaf(x2, -0x1.27e4fcp-22f, 0x1.a01a02p-16f);  // -1/10!, 1/8!
  c = std::fmaf(x2, c, -0x1.6c16c2p-10f);                      // -1/6!
  c = std::fmaf(x2, c, 0x1.555556p-5f);                        // 1/4!
  c = std::fmaf(x2, c, -0.5f);
  c = std::fmaf(x2, c, 1.0f);
  float sn = std::fmaf(x2, 0x1.71de3ap-19f, -0x1.a01a02p-13f);  // 1/9!, -1/7!
  sn = std::fmaf(x2, sn, 0x1.111112p-7f);                       // 1/5!
  sn = std::fmaf(x2, sn, -0x1.555556p-3f);                      // -1/3!
  const float x3 = x * x2;
  sn = std::fmaf(x3, sn, x);
  switch (q & 3u) {
    case 0: return c;
    case 1: return -sn;
    case 2: return -c;
    default: return sn;
  }
}

std::vector<double> box_muller(uint64_t seed, int level, int n) {
  std::vector<double> z(n);
  uint64_t key = stream_key(seed, level, 1);
  for (int i = 0; i < n; ++i) {
    const uint32_t k1 = unif24(key, 2 * (uint64_t)i);
    const uint32_t k2 = unif24(key, 2 * (uint64_t)i + 1);
    const float u1 = 1.0f - (float)k1 * 0x1p-24f;
    const float t = -2.0f * ln_f32(u1);
    z[i] = (double)(std::sqrt(t) * cos2pi_f32(k2));
  }
  return z;
}

// Steps 4-6: power basis K = [b, A b, ..., A^m b], QR of K by Householder reflections, and the
// least-squares problem min || beta e1 - R(:, 2:end) y || with beta = R(1,1).
// Reading (the paper is silent on breakdown): if a diagonal entry of R is negligible against
// its column (|R_cc| <= 1e-12 ||R(:,c)||, c >= 1), the Krylov space is exhausted at dimension c;
// only alpha_0..alpha_{c-1} are fitted and the rest are zero.  Returns the fitted count.
int poly_fit(const Csr& A, int m, const std::vector<double>& b, std::vector<double>& alpha) {
  int n = A.nrows, nc = m + 1;
  alpha.assign(m, 0.0);
  if (n == 0 || m <= 0) return 0;
  std::vector<std::vector<double>> K(nc, std::vector<double>(n));
  K[0] = b;
  for (int c = 1; c < nc; ++c) spmv(A, K[c - 1], K[c]);
  // Householder QR (columns of K overwritten).
  int kmax = std::min(n, nc);
  std::vector<double> Rm((size_t)nc * nc, 0.0);  // row-major upper triangle
  for (int k = 0; k < kmax; ++k) {
    double xn = 0.0;
    for (int r = k; r < n; ++r) xn += K[k][r] * K[k][r];
    xn = std::sqrt(xn);
    double a = (K[k][k] >= 0.0) ? -xn : xn;
    std::vector<double> v(K[k].begin() + k, K[k].end());
    v[0] -= a;
    double vn2 = 0.0;
    for (double t : v) vn2 += t * t;
    if (vn2 > 0.0) {
      for (int j = k; j < nc; ++j) {
        double s = 0.0;
        for (int r = k; r < n; ++r) s += v[r - k] * K[j][r];
        s = 2.0 * s / vn2;
        for (int r = k; r < n; ++r) K[j][r] -= s * v[r - k];
      }
    }
    for (int j = k; j < nc; ++j) Rm[(size_t)k * nc + j] = K[j][k];
  }
  auto R = [&](int i, int j) { return Rm[(size_t)i * nc + j]; };
  // breakdown detection
  int mf = m;
  for (int c = 1; c <= m; ++c) {
    double cn = 0.0;
    for (int r = 0; r <= c; ++r) cn += R(r, c) * R(r, c);
    cn = std::sqrt(cn);
    if (!(std::fabs(R(c, c)) > 1e-12 * cn)) { mf = c; break; }
  }
  // least squares on the (mf+1) x mf upper-Hessenberg H = R(0:mf, 1:mf) by Givens rotations
  std::vector<std::vector<double>> H(mf + 1, std::vector<double>(mf, 0.0));
  for (int i = 0; i <= mf; ++i)
    for (int j = 0; j < mf; ++j) H[i][j] = R(i, j + 1);
  std::vector<double> g(mf + 1, 0.0);
  g[0] = R(0, 0);
  for (int k = 0; k < mf; ++k) {
    double a = H[k][k], bb = H[k + 1][k];
    double d = std::hypot(a, bb);
    double cs = 1.0, sn = 0.0;
    if (d != 0.0) { cs = a / d; sn = bb / d; }
    for (int j = k; j < mf; ++j) {
      double t1 = H[k][j], t2 = H[k + 1][j];
      H[k][j] = cs * t1 + sn * t2;
      H[k + 1][j] = -sn * t1 + cs * t2;
    }
    double t1 = g[k], t2 = g[k + 1];
    g[k] = cs * t1 + sn * t2;
    g[k + 1] = -sn * t1 + cs * t2;
  }
  for (int i = mf - 1; i >= 0; --i) {
    double s = g[i];
    for (int j = i + 1; j < mf; ++j) s -= H[i][j] * alpha[j];
    alpha[i] = (H[i][i] != 0.0) ? s / H[i][i] : 0.0;
  }
  return mf;
}

// Pattern of A with the diagonal added if missing (values 0 there).
Csr with_diag(const Csr& A) {
  Csr B;
  B.nrows = A.nrows;
  B.ncols = A.ncols;
  B.rp.assign(1, 0);
  for (int i = 0; i < A.nrows; ++i) {
    bool has = false;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) has |= (A.ci[k] == i);
    bool placed = has;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      if (!placed && A.ci[k] > i) { B.ci.push_back(i); B.v.push_back(0.0); placed = true; }
      B.ci.push_back(A.ci[k]);
      B.v.push_back(A.v[k]);
    }
    if (!placed) { B.ci.push_back(i); B.v.push_back(0.0); }
    B.rp.push_back((int)B.ci.size());
  }
  return B;
}

// Steps 7-8 with fixed sparsity, eq. fixed_sparsity.  Reading: the powers are recursive,
// tilde(A^k) = P_T( tilde(A^{k-1}) A ), with T = pattern(A) plus the diagonal (first order) or the
// pattern of that pattern's square (second order, Section "AIRG": "enforcing the sparsity of
// A_ff^2"), so row i of each power needs only row i of the previous power and the rows of A in T_i.
//   tilde(A^1) = A on T (zeros where A has no entry)
//   tilde(A^k)_ij = sum_{l in T_i, ascending} tilde(A^{k-1})_il a_lj     (fma, a_lj absent skipped)
//   Ainv_ij = alpha_0 delta_ij + alpha_1 tilde(A^1)_ij + ... + alpha_{m-1} tilde(A^{m-1})_ij
// accumulated left to right with fma.

// Pattern of S*S (structural; S has its diagonal, so it contains pattern(S)), values: S's entries
// where S has one, 0 elsewhere.
Csr square_pattern(const Csr& S) {
  Csr T;
  T.nrows = S.nrows;
  T.ncols = S.ncols;
  T.rp.assign(1, 0);
  for (int i = 0; i < S.nrows; ++i) {
    std::map<int, double> cols;
    for (int k = S.rp[i]; k < S.rp[i + 1]; ++k) {
      const int l = S.ci[k];
      for (int q = S.rp[l]; q < S.rp[l + 1]; ++q) cols.emplace(S.ci[q], 0.0);
    }
    for (int k = S.rp[i]; k < S.rp[i + 1]; ++k) cols[S.ci[k]] = S.v[k];
    for (auto& kv : cols) {
      T.ci.push_back(kv.first);
      T.v.push_back(kv.second);
    }
    T.rp.push_back((int)T.ci.size());
  }
  return T;
}

Csr fixed_sparsity_inverse(const Csr& A0, const std::vector<double>& alpha, int order) {
  Csr S = with_diag(A0);
  Csr T = (order >= 2) ? square_pattern(S) : S;
  int m = (int)alpha.size();
  Csr Ainv = T;
  std::vector<double> prev = T.v, cur(T.v.size());
  for (int i = 0; i < T.nrows; ++i)
    for (int k = T.rp[i]; k < T.rp[i + 1]; ++k) {
      double acc = (T.ci[k] == i && m > 0) ? alpha[0] : 0.0;
      if (m > 1) acc = std::fma(alpha[1], prev[k], acc);
      Ainv.v[k] = acc;
    }
  for (int p = 2; p < m; ++p) {
    for (int i = 0; i < T.nrows; ++i)
      for (int k = T.rp[i]; k < T.rp[i + 1]; ++k) {
        int j = T.ci[k];
        double acc = 0.0;
        for (int q = T.rp[i]; q < T.rp[i + 1]; ++q) {
          int l = T.ci[q];
          if (has_entry(S, l, j)) acc = std::fma(prev[q], entry(S, l, j), acc);
        }
        cur[k] = acc;
      }
    for (int i = 0; i < T.nrows; ++i)
      for (int k = T.rp[i]; k < T.rp[i + 1]; ++k) Ainv.v[k] = std::fma(alpha[p], cur[k], Ainv.v[k]);
    std::swap(prev, cur);
  }
  return Ainv;
}

// ---------------------------------------------------------------------------------------------
// Sparse products with the relative row-wise infinity-norm drop (setup steps 9 and 11)
// ---------------------------------------------------------------------------------------------
// C = scale * (A B); entries with |c_ij| < tol * max_j |c_ij| are dropped (strict), the diagonal
// is kept when keep_diag.  Each c_ij accumulates a_il b_lj over ascending l with fma.
Csr spgemm(const Csr& A, const Csr& B, double scale, double tol, bool keep_diag) {
  Csr Cm;
  Cm.nrows = A.nrows;
  Cm.ncols = B.ncols;
  Cm.rp.assign(1, 0);
  for (int i = 0; i < A.nrows; ++i) {
    std::map<int, double> acc;
    for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      int l = A.ci[k];
      double a = A.v[k];
      for (int q = B.rp[l]; q < B.rp[l + 1]; ++q) {
        auto it = acc.find(B.ci[q]);
        double prev = (it == acc.end()) ? 0.0 : it->second;
        acc[B.ci[q]] = std::fma(a, B.v[q], prev);
      }
    }
    double mx = 0.0;
    for (auto& kv : acc) { kv.second = scale * kv.second; mx = std::max(mx, std::fabs(kv.second)); }
    double thr = tol * mx;
    for (auto& kv : acc) {
      if (std::fabs(kv.second) < thr && !(keep_diag && kv.first == i)) continue;
      Cm.ci.push_back(kv.first);
      Cm.v.push_back(kv.second);
    }
    Cm.rp.push_back((int)Cm.ci.size());
  }
  return Cm;
}

// ---------------------------------------------------------------------------------------------
// Hierarchy
// ---------------------------------------------------------------------------------------------
struct Level {
  Csr A;                     // level matrix, natural numbering
  std::vector<int8_t> cf;    // final CF splitting (empty on the coarsest level)
  std::vector<int8_t> cf_pmisr;
  std::vector<int> fidx, cidx, Fnat, Cnat;
  Csr Aff, Afc, Acf, Acc, Ainv, Z;
  std::vector<int> w;        // one-point prolongation: F index -> C index (-1: none)
  Csr W;                     // approximate ideal prolongator (n_f x n_c); empty for one-point P
  std::vector<double> alpha;
  int alpha_fitted = 0;
  int rounds = 0;
  double tau = INFINITY;
  bool coarsest = false;
};

struct Hier {
  Params p;
  std::vector<Level> lv;
  int top_nnz = 0;
};

void extract(Level& L) {
  const Csr& A = L.A;
  int n = A.nrows;
  L.fidx.assign(n, -1);
  L.cidx.assign(n, -1);
  L.Fnat.clear();
  L.Cnat.clear();
  for (int i = 0; i < n; ++i) {
    if (L.cf[i] == F) { L.fidx[i] = (int)L.Fnat.size(); L.Fnat.push_back(i); }
    else { L.cidx[i] = (int)L.Cnat.size(); L.Cnat.push_back(i); }
  }
  int nf = (int)L.Fnat.size(), nc = (int)L.Cnat.size();
  auto block = [&](const std::vector<int>& rows, bool colF, int ncols) {
    Csr B;
    B.nrows = (int)rows.size();
    B.ncols = ncols;
    B.rp.assign(1, 0);
    for (int i : rows) {
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        int j = A.ci[k];
        if ((L.cf[j] == F) != colF) continue;
        B.ci.push_back(colF ? L.fidx[j] : L.cidx[j]);
        B.v.push_back(A.v[k]);
      }
      B.rp.push_back((int)B.ci.size());
    }
    return B;
  };
  L.Aff = block(L.Fnat, true, nf);
  L.Afc = block(L.Fnat, false, nc);
  L.Acf = block(L.Cnat, true, nf);
  L.Acc = block(L.Cnat, false, nc);
}

// One-point prolongation (setup step 10, classical one-point operator).  Reading: each F-point
// takes the C-point among its strong dependencies with the largest |a_ij| (ties: smallest j),
// falling back to the largest |a_ij| over all nonzero C entries of the row; weight 1; no entry if
// the row has no C neighbour.
void one_point(Level& L, const std::vector<int8_t>& strong) {
  const Csr& A = L.A;
  L.w.assign(L.Fnat.size(), -1);
  for (size_t f = 0; f < L.Fnat.size(); ++f) {
    int i = L.Fnat[f];
    int best = -1;
    double bv = -1.0;
    for (int pass = 0; pass < 2 && best < 0; ++pass)
      for (int k = A.rp[i]; k < A.rp[i + 1]; ++k) {
        int j = A.ci[k];
        if (j == i || L.cf[j] != C || A.v[k] == 0.0) continue;
        if (pass == 0 && !strong[k]) continue;
        double a = std::fabs(A.v[k]);
        if (a > bv) { bv = a; best = j; }
      }
    L.w[f] = best >= 0 ? L.cidx[best] : -1;
  }
}

// Coarse matrix (setup step 11): A_c = R (A P), P = [W; I], R = [Z I] in natural numbering.  W is
// the approximate ideal prolongator when the level has one, else the one-point operator.
Csr coarse_matrix(const Level& L, double drop) {
  const Csr& A = L.A;
  int n = A.nrows, nc = (int)L.Cnat.size();
  Csr P;
  P.nrows = n;
  P.ncols = nc;
  P.rp.assign(1, 0);
  const bool ideal = L.W.nrows > 0;
  for (int i = 0; i < n; ++i) {
    if (ideal && L.cf[i] == F) {
      int f = L.fidx[i];
      for (int k = L.W.rp[f]; k < L.W.rp[f + 1]; ++k) { P.ci.push_back(L.W.ci[k]); P.v.push_back(L.W.v[k]); }
    } else {
      int c = (L.cf[i] == C) ? L.cidx[i] : L.w[L.fidx[i]];
      if (c >= 0) { P.ci.push_back(c); P.v.push_back(1.0); }
    }
    P.rp.push_back((int)P.ci.size());
  }
  Csr AP = spgemm(A, P, 1.0, 0.0, false);
  Csr R;
  R.nrows = nc;
  R.ncols = n;
  R.rp.assign(1, 0);
  for (int c = 0; c < nc; ++c) {
    std::vector<std::pair<int, double>> row;
    for (int k = L.Z.rp[c]; k < L.Z.rp[c + 1]; ++k) row.push_back({L.Fnat[L.Z.ci[k]], L.Z.v[k]});
    row.push_back({L.Cnat[c], 1.0});
    std::sort(row.begin(), row.end());
    for (auto& e : row) { R.ci.push_back(e.first); R.v.push_back(e.second); }
    R.rp.push_back((int)R.ci.size());
  }
  return spgemm(R, AP, 1.0, drop, true);
}

// forced[l] (when l < forced.size()) is level l's CF splitting, taken as given instead of computed
// (setup re-use); the strength flags the one-point prolongator reads are still computed.  Returns
// false if a forced splitting does not have its level's size.
bool build(Hier& H, const Csr& A0, const std::vector<std::vector<int8_t>>& forced = {}) {
  const Params& p = H.p;
  H.top_nnz = A0.nnz();
  Csr A = A0;
  int m = p.poly_order + 1, mc = p.coarse_poly_order + 1;
  for (int l = 0;; ++l) {
    Level L;
    L.A = A;
    int n = A.nrows;
    bool coarsest = (n <= p.coarse_size) || (n < m) || (l == p.max_levels - 1);
    std::vector<int8_t> strong;
    if (!coarsest && l < (int)forced.size()) {
      if ((int)forced[l].size() != n) return false;
      L.cf = forced[l];
      L.cf_pmisr = forced[l];
      strong = strength(A, p.strong_threshold);
      long nf = std::count(L.cf.begin(), L.cf.end(), (int8_t)F);
      if (nf == 0 || nf == n) { coarsest = true; L.cf.clear(); L.cf_pmisr.clear(); }
    } else if (!coarsest) {
      CfDetail d = cf_split(A, p, l);
      L.cf = d.cf;
      L.cf_pmisr = d.cf_pmisr;
      L.rounds = d.rounds;
      L.tau = d.tau;
      strong = d.strong;
      long nf = std::count(L.cf.begin(), L.cf.end(), (int8_t)F);
      if (nf == 0 || nf == n) { coarsest = true; L.cf.clear(); L.cf_pmisr.clear(); }
    }
    if (coarsest) {
      L.coarsest = true;
      std::vector<double> bt = box_muller(p.seed, l, n);
      L.alpha_fitted = poly_fit(A, mc, bt, L.alpha);
      L.Ainv = fixed_sparsity_inverse(A, L.alpha, 1);
      H.lv.push_back(std::move(L));
      return true;
    }
    extract(L);
    std::vector<double> bt = box_muller(p.seed, l, (int)L.Fnat.size());
    L.alpha_fitted = poly_fit(L.Aff, m, bt, L.alpha);
    L.Ainv = fixed_sparsity_inverse(L.Aff, L.alpha, p.sparsity_order);
    L.Z = spgemm(L.Acf, L.Ainv, -1.0, p.drop_R, false);
    one_point(L, strong);
    // setup step 10's alternative: the prolongator's counterpart of Z (eq. prolong),
    // W = -Ainv A_fc, with Z's relative drop tolerance
    if (p.ideal_prolong) L.W = spgemm(L.Ainv, L.Afc, -1.0, p.drop_R, false);
    Csr Ac = coarse_matrix(L, p.drop_Ac);
    H.lv.push_back(std::move(L));
    A = std::move(Ac);
  }
}

// ---------------------------------------------------------------------------------------------
// Solve phase
// ---------------------------------------------------------------------------------------------
// V-cycle (Section "Results"): zero initial guess, restriction with R = [Z I], recursion,
// one-point prolongation, then n_smooth_up F-point smooths x_F += Ainv (b_F - A_ff x_F - A_fc x_C);
// no down-smoothing.  Coarsest level: coarse_iters iterations of x += Ainv_L (b - A_L x).
// The stationary polynomial applied without assembling it (Section "AIRG" names this alternative
// to the fixed-sparsity matrix): t = q(A) r = sum_{k<m} alpha_k A^k r, from the power basis
// v_0 = r, v_k = A v_{k-1}.
void poly_apply(const Csr& A, const std::vector<double>& alpha, const std::vector<double>& r, std::vector<double>& t) {
  int n = A.nrows;
  t.assign(n, 0.0);
  std::vector<double> v = r, Av;
  for (size_t k = 0; k < alpha.size(); ++k) {
    if (k > 0) {
      spmv(A, v, Av);
      v.swap(Av);
    }
    for (int i = 0; i < n; ++i) t[i] += alpha[k] * v[i];
  }
}

void vcycle(const Hier& H, int l, const std::vector<double>& b, std::vector<double>& x) {
  const Level& L = H.lv[l];
  const bool mf = H.p.matrix_free != 0;
  int n = L.A.nrows;
  x.assign(n, 0.0);
  if (L.coarsest) {
    std::vector<double> r(n), t;
    for (int it = 0; it < H.p.coarse_iters; ++it) {
      spmv(L.A, x, t);
      for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
      if (mf) poly_apply(L.A, L.alpha, r, t);
      else spmv(L.Ainv, r, t);
      for (int i = 0; i < n; ++i) x[i] += t[i];
    }
    return;
  }
  int nf = (int)L.Fnat.size(), nc = (int)L.Cnat.size();
  std::vector<double> bF(nf), bC(nc), xF(nf, 0.0), xC, t;
  for (int f = 0; f < nf; ++f) bF[f] = b[L.Fnat[f]];
  for (int c = 0; c < nc; ++c) bC[c] = b[L.Cnat[c]];
  spmv(L.Z, bF, t);
  for (int c = 0; c < nc; ++c) bC[c] += t[c];
  vcycle(H, l + 1, bC, xC);
  if (L.W.nrows > 0) spmv(L.W, xC, xF);  // x_F = W x_C
  else
    for (int f = 0; f < nf; ++f) xF[f] = (L.w[f] >= 0) ? xC[L.w[f]] : 0.0;
  std::vector<double> r(nf), t2;
  for (int s = 0; s < H.p.n_smooth_up; ++s) {
    spmv(L.Aff, xF, t);
    spmv(L.Afc, xC, t2);
    for (int f = 0; f < nf; ++f) r[f] = bF[f] - t[f] - t2[f];
    if (mf) poly_apply(L.Aff, L.alpha, r, t);
    else spmv(L.Ainv, r, t);
    for (int f = 0; f < nf; ++f) xF[f] += t[f];
  }
  for (int f = 0; f < nf; ++f) x[L.Fnat[f]] = xF[f];
  for (int c = 0; c < nc; ++c) x[L.Cnat[c]] = xC[c];
}

struct SolveOut {
  int iters = 0;
  double relres = 0.0;
  int status = 0;  // 0 converged, 1 not converged, -4 nan
};

// Right-preconditioned FGMRES(restart) with classical Gram-Schmidt applied twice (CGS2).
// Convergence: Givens estimate |g_{j+1}| / ||b|| <= rtol, confirmed by the true residual before
// returning (restart otherwise).  An iteration is one preconditioner application.
// precond = 0 applies no preconditioner (identity).
SolveOut fgmres(const Hier* H, const Csr& A, const std::vector<double>& b, std::vector<double>& x,
                int restart, int max_it, double rtol, std::vector<double>* hist, bool precond) {
  SolveOut o;
  int n = A.nrows;
  double bn = nrm2(b);
  if (bn == 0.0) { x.assign(n, 0.0); o.relres = 0.0; return o; }
  std::vector<double> r(n), t;
  auto true_res = [&]() {
    spmv(A, x, t);
    for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
    return nrm2(r);
  };
  double beta = true_res();
  o.relres = beta / bn;
  if (hist) hist->push_back(o.relres);
  while (true) {
    if (!(o.relres == o.relres)) { o.status = -4; return o; }
    if (o.relres <= rtol) return o;
    if (o.iters >= max_it) { o.status = 1; return o; }
    std::vector<std::vector<double>> V(1, std::vector<double>(n)), Zs;
    for (int i = 0; i < n; ++i) V[0][i] = r[i] / beta;
    std::vector<std::vector<double>> Hh;  // columns
    std::vector<double> cs, sn, g{beta};
    int j = 0;
    for (; j < restart && o.iters < max_it; ++j) {
      std::vector<double> z;
      if (precond) vcycle(*H, 0, V[j], z); else z = V[j];
      Zs.push_back(z);
      std::vector<double> w;
      spmv(A, z, w);
      std::vector<double> h(j + 2, 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        std::vector<double> hp(j + 1);
        for (int i = 0; i <= j; ++i) hp[i] = dot(V[i], w);
        for (int i = 0; i <= j; ++i)
          for (int q = 0; q < n; ++q) w[q] -= hp[i] * V[i][q];
        for (int i = 0; i <= j; ++i) h[i] += hp[i];
      }
      h[j + 1] = nrm2(w);
      for (int i = 0; i < j; ++i) {
        double t1 = h[i], t2 = h[i + 1];
        h[i] = cs[i] * t1 + sn[i] * t2;
        h[i + 1] = -sn[i] * t1 + cs[i] * t2;
      }
      double d = std::hypot(h[j], h[j + 1]);
      double c_ = 1.0, s_ = 0.0;
      if (d != 0.0) { c_ = h[j] / d; s_ = h[j + 1] / d; }
      double hj1 = h[j + 1];
      h[j] = c_ * h[j] + s_ * h[j + 1];
      h[j + 1] = 0.0;
      cs.push_back(c_);
      sn.push_back(s_);
      g.push_back(-s_ * g[j]);
      g[j] = c_ * g[j];
      Hh.push_back(h);
      o.iters++;
      double est = std::fabs(g[j + 1]) / bn;
      if (hist) hist->push_back(est);
      if (est <= rtol || hj1 == 0.0 || !(est == est)) { ++j; break; }
      V.push_back(std::vector<double>(n));
      for (int q = 0; q < n; ++q) V[j + 1][q] = w[q] / hj1;
    }
    int k = j;
    std::vector<double> y(k);
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int q = i + 1; q < k; ++q) s -= Hh[q][i] * y[q];
      y[i] = s / Hh[i][i];
    }
    for (int i = 0; i < k; ++i)
      for (int q = 0; q < n; ++q) x[q] += y[i] * Zs[i][q];
    beta = true_res();
    o.relres = beta / bn;
  }
}

// Undamped Richardson (Section "Results"): x += M (b - A x).
SolveOut richardson(const Hier& H, const std::vector<double>& b, std::vector<double>& x, int max_it,
                    double rtol, std::vector<double>* hist) {
  SolveOut o;
  const Csr& A = H.lv[0].A;
  int n = A.nrows;
  double bn = nrm2(b);
  if (bn == 0.0) { x.assign(n, 0.0); return o; }
  std::vector<double> r(n), t, z;
  while (true) {
    spmv(A, x, t);
    for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];
    o.relres = nrm2(r) / bn;
    if (hist) hist->push_back(o.relres);
    if (!(o.relres == o.relres)) { o.status = -4; return o; }
    if (o.relres <= rtol) return o;
    if (o.iters >= max_it) { o.status = 1; return o; }
    vcycle(H, 0, r, z);
    for (int i = 0; i < n; ++i) x[i] += z[i];
    o.iters++;
  }
}

// Dense LU with partial pivoting (the plain definition x* = A^-1 b for tiny systems).
int dense_solve(int n, std::vector<double> M, std::vector<double> b, std::vector<double>& x) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(M[(size_t)i * n + k]) > std::fabs(M[(size_t)p * n + k])) p = i;
    if (M[(size_t)p * n + k] == 0.0) return -1;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(M[(size_t)k * n + j], M[(size_t)p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      double f = M[(size_t)i * n + k] / M[(size_t)k * n + k];
      M[(size_t)i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= M[(size_t)i * n + j] * x[j];
    x[i] = s / M[(size_t)i * n + i];
  }
  return 0;
}

bool valid_csr(int n, const int* rp, const int* ci) {
  if (n < 0 || !rp || rp[0] != 0) return false;
  for (int i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return false;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < 0 || ci[k] >= n) return false;
      if (k > rp[i] && ci[k] <= ci[k - 1]) return false;
    }
  }
  return true;
}

Params to_params(const double* dp, const long long* ip) {
  Params p;
  p.strong_threshold = dp[0];
  p.ddc_fraction = dp[1];
  p.drop_R = dp[2];
  p.drop_Ac = dp[3];
  p.pmisr_max_loops = (int)ip[0];
  p.poly_order = (int)ip[1];
  p.coarse_poly_order = (int)ip[2];
  p.coarse_iters = (int)ip[3];
  p.coarse_size = (int)ip[4];
  p.max_levels = (int)ip[5];
  p.n_smooth_up = (int)ip[6];
  p.one_point_weighted = (int)ip[7];
  p.seed = (uint64_t)ip[8];
  p.sparsity_order = (int)ip[9];
  p.matrix_free = (int)ip[10];
  p.ideal_prolong = (int)ip[11];
  return p;
}

void copy_csr(const Csr& A, int* rp, int* ci, double* v) {
  if (rp) std::copy(A.rp.begin(), A.rp.end(), rp);
  if (ci) std::copy(A.ci.begin(), A.ci.end(), ci);
  if (v) std::copy(A.v.begin(), A.v.end(), v);
}

}  // namespace

// =============================================================================================
// C API (loaded by the tests through ctypes).  Parameters travel as two flat arrays:
//   dp = {strong_threshold, ddc_fraction, drop_R, drop_Ac}
//   ip = {pmisr_max_loops, poly_order, coarse_poly_order, coarse_iters, coarse_size, max_levels,
//         n_smooth_up, one_point_weighted, seed}
// Return codes: 0 ok, -1 bad argument / CSR, -2 singular, 1 not converged, -4 NaN.
// =============================================================================================
extern "C" {

// Threads of the SpMV row loop (at least 1); returns the previous count.
int oracle_set_threads(int t) {
  const int prev = g_threads;
  g_threads = t < 1 ? 1 : t;
  return prev;
}

int oracle_setup(int n, const int* rp, const int* ci, const double* v, const double* dp, const long long* ip,
                 void** out) {
  if (!out || !valid_csr(n, rp, ci)) return -1;
  Hier* H = new (std::nothrow) Hier;
  if (!H) return -1;
  H->p = to_params(dp, ip);
  build(*H, make_csr(n, n, rp, ci, v));
  *out = H;
  return 0;
}

// Setup with the CF splittings of the first nforced levels given (cfs[l]: cf_len[l] entries,
// 1 = F, 2 = C): the setup re-use of the library, restated.  Returns -2 if a splitting does not
// have its level's size.
int oracle_setup_forced(int n, const int* rp, const int* ci, const double* v, const double* dp, const long long* ip,
                        int nforced, const int8_t* const* cfs, const int* cf_len, void** out) {
  if (!out || !valid_csr(n, rp, ci) || nforced < 0) return -1;
  std::vector<std::vector<int8_t>> forced(nforced);
  for (int l = 0; l < nforced; ++l) forced[l].assign(cfs[l], cfs[l] + cf_len[l]);
  Hier* H = new (std::nothrow) Hier;
  if (!H) return -1;
  H->p = to_params(dp, ip);
  if (!build(*H, make_csr(n, n, rp, ci, v), forced)) {
    delete H;
    return -2;
  }
  *out = H;
  return 0;
}

void oracle_free(void* h) { delete (Hier*)h; }

int oracle_num_levels(void* h) { return (int)((Hier*)h)->lv.size(); }

// info[0..11] = n, nnz(A), n_f, n_c, nnz(Aff), nnz(Afc), nnz(Ainv), nnz(Z), coarsest, pmisr rounds,
//              alpha_fitted, nnz(Acf)
int oracle_level_info(void* h, int l, long long* info, double* tau) {
  Hier* H = (Hier*)h;
  if (l < 0 || l >= (int)H->lv.size()) return -1;
  const Level& L = H->lv[l];
  info[0] = L.A.nrows;
  info[1] = L.A.nnz();
  info[2] = (long long)L.Fnat.size();
  info[3] = (long long)L.Cnat.size();
  info[4] = L.Aff.nnz();
  info[5] = L.Afc.nnz();
  info[6] = L.Ainv.nnz();
  info[7] = L.Z.nnz();
  info[8] = L.coarsest;
  info[9] = L.rounds;
  info[10] = L.alpha_fitted;
  info[11] = L.Acf.nnz();
  info[12] = L.W.nnz();
  if (tau) *tau = L.tau;
  return 0;
}

// which: 0 A, 1 Aff, 2 Afc, 3 Acf, 4 Acc, 5 Ainv, 6 Z, 7 W  (CSR export; call with the sizes from
// oracle_level_info).
int oracle_export_csr(void* h, int l, int which, int* rp, int* ci, double* v) {
  Hier* H = (Hier*)h;
  if (l < 0 || l >= (int)H->lv.size()) return -1;
  const Level& L = H->lv[l];
  const Csr* M = nullptr;
  switch (which) {
    case 0: M = &L.A; break;
    case 1: M = &L.Aff; break;
    case 2: M = &L.Afc; break;
    case 3: M = &L.Acf; break;
    case 4: M = &L.Acc; break;
    case 5: M = &L.Ainv; break;
    case 6: M = &L.Z; break;
    case 7: M = &L.W; break;
    default: return -1;
  }
  copy_csr(*M, rp, ci, v);
  return 0;
}

// cf (int8, n; 1 = F, 2 = C), cf before DDC, w (int32, n_f), alpha (m)
int oracle_export_vectors(void* h, int l, int8_t* cf, int8_t* cf_pmisr, int* w, double* alpha) {
  Hier* H = (Hier*)h;
  if (l < 0 || l >= (int)H->lv.size()) return -1;
  const Level& L = H->lv[l];
  if (cf) std::copy(L.cf.begin(), L.cf.end(), cf);
  if (cf_pmisr) std::copy(L.cf_pmisr.begin(), L.cf_pmisr.end(), cf_pmisr);
  if (w) std::copy(L.w.begin(), L.w.end(), w);
  if (alpha) std::copy(L.alpha.begin(), L.alpha.end(), alpha);
  return 0;
}

// outer: 0 FGMRES, 1 Richardson, 2 unpreconditioned GMRES.  x: in x0, out solution.
int oracle_solve(void* h, const double* b, double* x, int outer, int restart, int max_it, double rtol,
                 int* iters, double* relres, double* hist, int hist_len) {
  Hier* H = (Hier*)h;
  int n = H->lv[0].A.nrows;
  std::vector<double> bb(b, b + n), xx(x, x + n), hs;
  SolveOut o;
  if (outer == 1) o = richardson(*H, bb, xx, max_it, rtol, &hs);
  else o = fgmres(H, H->lv[0].A, bb, xx, restart, max_it, rtol, &hs, outer == 0);
  std::copy(xx.begin(), xx.end(), x);
  if (iters) *iters = o.iters;
  if (relres) *relres = o.relres;
  if (hist)
    for (int i = 0; i < hist_len && i < (int)hs.size(); ++i) hist[i] = hs[i];
  return o.status;
}

// One V-cycle from zero: x = M b.
int oracle_vcycle(void* h, const double* b, double* x) {
  Hier* H = (Hier*)h;
  int n = H->lv[0].A.nrows;
  std::vector<double> bb(b, b + n), xx;
  vcycle(*H, 0, bb, xx);
  std::copy(xx.begin(), xx.end(), x);
  return 0;
}

// CF splitting of one matrix, with every intermediate: strong flags (nnz), weights w (n),
// cf after PMISR (n), theta (n), final cf (n), tau, rounds.
int oracle_cf_split(int n, const int* rp, const int* ci, const double* v, const double* dp, const long long* ip,
                    int level, int8_t* strong, double* w, int8_t* cf_pmisr, double* theta, int8_t* cf,
                    double* tau, int* rounds) {
  if (!valid_csr(n, rp, ci)) return -1;
  Params p = to_params(dp, ip);
  CfDetail d = cf_split(make_csr(n, n, rp, ci, v), p, level);
  if (strong) std::copy(d.strong.begin(), d.strong.end(), strong);
  if (w) std::copy(d.w.begin(), d.w.end(), w);
  if (cf_pmisr) std::copy(d.cf_pmisr.begin(), d.cf_pmisr.end(), cf_pmisr);
  if (theta) std::copy(d.theta.begin(), d.theta.end(), theta);
  if (cf) std::copy(d.cf.begin(), d.cf.end(), cf);
  if (tau) *tau = d.tau;
  if (rounds) *rounds = d.rounds;
  return 0;
}

// PMISR alone on a given strong-flag array and weight vector (for brute-force pins).
int oracle_pmisr(int n, const int* rp, const int* ci, const int8_t* strong, const double* w, int max_loops,
                 int8_t* cf, int* rounds) {
  Csr A;
  A.nrows = A.ncols = n;
  A.rp.assign(rp, rp + n + 1);
  A.ci.assign(ci, ci + rp[n]);
  A.v.assign(rp[n], 1.0);
  std::vector<int8_t> s(strong, strong + rp[n]);
  Graph g = sym_graph(A, s);
  std::vector<double> ww(w, w + n);
  std::vector<int8_t> out = pmisr(g, ww, max_loops, rounds);
  std::copy(out.begin(), out.end(), cf);
  return 0;
}

// DDC alone on a given CF splitting.
int oracle_ddc(int n, const int* rp, const int* ci, const double* v, const int8_t* cf_in, double fraction,
               int8_t* cf_out, double* theta, double* tau) {
  Csr A = make_csr(n, n, rp, ci, v);
  std::vector<int8_t> c(cf_in, cf_in + n);
  std::vector<double> th;
  std::vector<int8_t> out = ddc(A, c, fraction, tau, &th);
  std::copy(out.begin(), out.end(), cf_out);
  if (theta) std::copy(th.begin(), th.end(), theta);
  return 0;
}

// Polynomial coefficients for matrix A and right-hand side b (b == null: Box-Muller from seed,
// level).  Returns the fitted count.
int oracle_poly_fit(int n, const int* rp, const int* ci, const double* v, int m, const double* b,
                    unsigned long long seed, int level, double* alpha) {
  Csr A = make_csr(n, n, rp, ci, v);
  std::vector<double> bb = b ? std::vector<double>(b, b + n) : box_muller(seed, level, n);
  std::vector<double> al;
  int mf = poly_fit(A, m, bb, al);
  std::copy(al.begin(), al.end(), alpha);
  return mf;
}

int oracle_box_muller(unsigned long long seed, int level, int n, double* z) {
  std::vector<double> r = box_muller(seed, level, n);
  std::copy(r.begin(), r.end(), z);
  return 0;
}

int oracle_unif24(unsigned long long seed, int level, int stream, int n, unsigned int* r) {
  uint64_t key = stream_key(seed, level, stream);
  for (int i = 0; i < n; ++i) r[i] = unif24(key, (uint64_t)i);
  return 0;
}
int oracle_unif01(unsigned long long seed, int level, int stream, int n, double* r) {
  uint64_t key = stream_key(seed, level, stream);
  for (int i = 0; i < n; ++i) r[i] = unif01(key, (uint64_t)i);
  return 0;
}

// Fixed-sparsity approximate inverse on pattern(A) plus diagonal.  Output sized with
// oracle_pattern_nnz.
int oracle_pattern_nnz(int n, const int* rp, const int* ci) {
  int add = 0;
  for (int i = 0; i < n; ++i) {
    bool has = false;
    for (int k = rp[i]; k < rp[i + 1]; ++k) has |= (ci[k] == i);
    add += !has;
  }
  return rp[n] + add;
}
int oracle_fixed_sparsity_inverse(int n, const int* rp, const int* ci, const double* v, int m,
                                  const double* alpha, int order, int* orp, int* oci, double* ov) {
  Csr A = make_csr(n, n, rp, ci, v);
  std::vector<double> al(alpha, alpha + m);
  Csr R = fixed_sparsity_inverse(A, al, order);
  if (!oci) {  // sizes only
    std::copy(R.rp.begin(), R.rp.end(), orp);
    return 0;
  }
  copy_csr(R, orp, oci, ov);
  return 0;
}

// Generic product with drop; two-call protocol: first with orp only (sizes), then full.
int oracle_spgemm(int ar, int ac, const int* arp, const int* aci, const double* av, int bc, const int* brp,
                  const int* bci, const double* bv, double scale, double tol, int keep_diag, int* orp,
                  int* oci, double* ov) {
  Csr A = make_csr(ar, ac, arp, aci, av);
  Csr B = make_csr(ac, bc, brp, bci, bv);
  copy_csr(spgemm(A, B, scale, tol, keep_diag != 0), orp, oci, ov);
  return 0;
}

int oracle_spmv(int n, const int* rp, const int* ci, const double* v, const double* x, double* y) {
  Csr A = make_csr(n, n, rp, ci, v);
  std::vector<double> xx(x, x + n), yy;
  spmv(A, xx, yy);
  std::copy(yy.begin(), yy.end(), y);
  return 0;
}

int oracle_dense_solve(int n, const int* rp, const int* ci, const double* v, const double* b, double* x) {
  std::vector<double> M((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = rp[i]; k < rp[i + 1]; ++k) M[(size_t)i * n + ci[k]] += v[k];
  std::vector<double> bb(b, b + n), xx;
  int rc = dense_solve(n, M, bb, xx);
  if (rc == 0) std::copy(xx.begin(), xx.end(), x);
  return rc == 0 ? 0 : -2;
}

// Hierarchy complexities (Section "Strong tolerances", eq. mat_store):
// out[0] grid complexity, out[1] operator complexity, out[2] storage complexity.
int oracle_complexities(void* h, double* out) {
  Hier* H = (Hier*)h;
  double n0 = H->lv[0].A.nrows, z0 = H->lv[0].A.nnz();
  double gs = 0, os = 0, st = 0;
  for (size_t l = 0; l < H->lv.size(); ++l) {
    const Level& L = H->lv[l];
    gs += L.A.nrows;
    os += L.A.nnz();
    if (L.coarsest) st += L.Ainv.nnz() + (H->p.coarse_iters > 1 ? L.A.nnz() : 0);
    else {
      long nP = 0;
      for (int w : L.w) nP += (w >= 0);
      nP += (long)L.Cnat.size();
      st += L.Ainv.nnz() + L.Aff.nnz() + L.Afc.nnz() + (L.Z.nnz() + (long)L.Cnat.size()) + nP;
    }
  }
  out[0] = gs / n0;
  out[1] = os / z0;
  out[2] = st / z0;
  return 0;
}

}  // extern "C"
