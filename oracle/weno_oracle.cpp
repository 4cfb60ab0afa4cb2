// weno_oracle.cpp -- plain, slow, single-threaded CPU oracle of WENO-ZA6.
//
// TEST INFRASTRUCTURE ONLY: the reference that the CUDA path is checked
// against.  Only the tests, the smoke check and the benchmark's CPU-baseline
// leg load it.  It shares no code with the CUDA library.  Build flags:
// g++ -O2 -ffp-contract=off (no fused multiply-add, so results are the same
// on every host).
//
// Every routine follows the paper (Gu, Wang, Don, Jung, arXiv 2603.26272) step
// by step, in the paper's order and notation, with the printed coefficient
// tables; nothing is fused or reordered.  Where the paper is silent the
// reading taken is stated at the routine.
//
// Parity pins: every function here is pinned by a test in tests/test_oracle_*.py
// (coefficients re-derived from eq. (15) in rational arithmetic, Tables 3 and 4,
// the smooth-data collapse to the linear flux, the discontinuity suppression of
// Section 2.2, affine invariance, conservation, mirror symmetry, 1D/2D
// consistency, sixth-order convergence and exact Riemann solutions).
#include "weno_oracle.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Real types.  double everywhere; a quadruple-precision type only for the
// operator-accuracy experiment of Tables 3 and 4, whose smallest entries lie
// below double rounding.
// ---------------------------------------------------------------------------
#if defined(__x86_64__)
typedef __float128 quad;
#elif defined(__aarch64__)
typedef long double quad;  // IEEE binary128 on AArch64 Linux
#else
typedef long double quad;
#endif

template <class R> R r_abs(R x) { return x < R(0) ? -x : x; }

// Summation order of the final sums (the convex combination of eq. (14) and
// its normaliser, the projections on L and the back-projection on R): k-th
// term of n.  The stock build adds in index order; the build with
// ORA_REVERSED_SUMS adds the same terms in the opposite order, a second
// rounding of the same arithmetic that shows how much a run amplifies
// rounding differences.
#ifndef ORA_REVERSED_SUMS
#define ORA_REVERSED_SUMS 0
#endif
inline int sum_ix(int k, int n) { return ORA_REVERSED_SUMS ? n - 1 - k : k; }

// Square root: std::sqrt for double; for quad, Newton's iteration
// y <- (y + x/y)/2 started from the double square root (quadratic convergence:
// three steps take 53 correct bits well past 113).
template <class R> R r_sqrt(R x);
template <> double r_sqrt<double>(double x) { return std::sqrt(x); }
template <> quad r_sqrt<quad>(quad x) {
  if (!(x > 0)) return quad(0);
  quad y = (quad)std::sqrt((double)x);
  for (int it = 0; it < 3; ++it) y = (y + x / y) / 2;
  return y;
}

// x^p for the power parameter of eq. (21).
template <class R> R r_pow(R x, double p);
template <> double r_pow<double>(double x, double p) {
  if (p == 1.0) return x;
  return std::pow(x, p);
}
template <> quad r_pow<quad>(quad x, double p) {
  if (p == 1.0) return x;
  if (p == 1.5) return x * r_sqrt<quad>(x);
  if (p == 2.0) return x * x;
  return (quad)std::pow((double)x, p);  // not used by the experiments
}

// exp(y) by its Taylor series, summed until the terms vanish (|y| <= 1 here).
template <class R> R r_exp(R y) {
  R s = 1, t = 1;
  for (int k = 1; k < 80; ++k) {
    t = t * y / R(k);
    s = s + t;
  }
  return s;
}

// ---------------------------------------------------------------------------
// Section 3: coefficients of the sixth-order scheme (r = 3), as printed.
// ---------------------------------------------------------------------------
// eq. (10): c_6 = (1, -8, 37, 37, -8, 1) / 60 on S^6.
const int C6_NUM[6] = {1, -8, 37, 37, -8, 1};
const int C6_DEN = 60;
// eq. (11): c_k on the 3-point substencils S_0..S_3, denominators 6.
const int CK_NUM[4][3] = {{2, -7, 11}, {-1, 5, 2}, {2, 5, -1}, {11, -7, 2}};
const int CK_DEN = 6;
// eq. (12)/(13): ideal weights d = (1, 9, 9, 1) / 20 = C(3,k)^2 / C(6,3).
const int D_NUM[4] = {1, 9, 9, 1};
const int D_DEN = 20;
// eq. (15) for r = 3: smoothness matrices, denominators 6.  B_2 = rev(B_0).
const int B0_NUM[3][3] = {{8, -19, 11}, {-19, 50, -31}, {11, -31, 20}};
const int B1_NUM[3][3] = {{8, -13, 5}, {-13, 26, -13}, {5, -13, 8}};
const int BD_NUM[3][3] = {{44, -73, 29}, {-73, 122, -49}, {29, -49, 20}};
const int B_DEN = 6;
// eq. (17): c_tau = (-1, 5, -10, 10, -5, 1).
const int CTAU[6] = {-1, 5, -10, 10, -5, 1};

// rev(.) of a 3x3 matrix: reverse both index orders.
int b2_num(int a, int b) { return B0_NUM[2 - a][2 - b]; }

// <f, B f> with B = Bnum / 6 (eq. (15) in the printed matrix form).
template <class R> R quad_form(const int Bnum[3][3], const R *f) {
  R s = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) s = s + f[a] * R(Bnum[a][b]) * f[b];
  return s / R(B_DEN);
}
template <class R> R quad_form_b2(const R *f) {
  R s = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) s = s + f[a] * R(b2_num(a, b)) * f[b];
  return s / R(B_DEN);
}

// ---------------------------------------------------------------------------
// WENO-ZA6 reconstruction of the positive flux at x_{i+1/2} (Section 3).
// Input f[0..5] = f_{i-2}, ..., f_{i+3} (the stencil S^6 of eq. (7)).
// The negative flux uses the same routine on the mirrored stencil
// (f_{i+3}, ..., f_{i-2}), Section 2 after eq. (6).
// ---------------------------------------------------------------------------
template <class R> struct ZA6Out {
  R fk[4];     // candidate fluxes f_hat^k, eq. (11)
  R beta[5];   // beta_0, beta_1, beta_2, beta_d, beta_3
  R tau;       // eq. (17)
  R mu;        // eq. (22) (1 when ai = 0)
  R omega[4];  // eq. (19)
  R fhat;      // eq. (14)
};

template <class R>
void za6_flux(const R f[6], R eps, R mu0, double p, int ai, ZA6Out<R> *o) {
  // eq. (11): f_hat^k = <c_k, f_k>, f_k = (f_{i-2+k}, f_{i-1+k}, f_{i+k}).
  for (int k = 0; k < 4; ++k) {
    R s = 0;
    for (int m = 0; m < 3; ++m) s = s + R(CK_NUM[k][m]) * f[k + m];
    o->fk[k] = s / R(CK_DEN);
  }
  // The indicators of eqs. (15), (17) and the descaler of eq. (22) depend on
  // f only through its variation: every row of every B_k sums to zero, and so
  // do c_tau and the deviations of eq. (22).  They are therefore evaluated on
  // shifted data -- each beta_k on f_k minus its own first entry, tau and mu
  // on f minus the stencil mean -- which are the same quantities with
  // rounding relative to the variation rather than to the level.  (Unshifted,
  // a flat substencil at a level c gives a rounding residual of either sign
  // of size ~1e-16 c^2 instead of 0, and beta_k + eps mu^2 < 0 then wrecks
  // the weights.)
  R mean = 0;
  for (int j = 0; j < 6; ++j) mean = mean + f[j];
  mean = mean / R(6);
  R g[6];
  for (int j = 0; j < 6; ++j) g[j] = f[j] - mean;
  R sk[4][3];
  for (int k = 0; k < 4; ++k)
    for (int m = 0; m < 3; ++m) sk[k][m] = f[k + m] - f[k];
  // eq. (15): local indicators beta_k = <f_k, B_k f_k>, k in {0, 1, 2, d}.
  R b0 = quad_form<R>(B0_NUM, sk[0]);
  R b1 = quad_form<R>(B1_NUM, sk[1]);
  R b2 = quad_form_b2<R>(sk[2]);
  R bd = quad_form<R>(BD_NUM, sk[3]);
  // eq. (16): the downwind indicator is the mean of all r + 1 = 4 indicators.
  R b3 = (b0 + b1 + b2 + bd) / R(4);
  o->beta[0] = b0;
  o->beta[1] = b1;
  o->beta[2] = b2;
  o->beta[3] = bd;
  o->beta[4] = b3;
  // eq. (17): tau = <c_tau, f^6>^2.
  R t = 0;
  for (int j = 0; j < 6; ++j) t = t + R(CTAU[j]) * g[j];
  R tau = t * t;
  o->tau = tau;
  // eq. (22): affine-invariant descaler mu[f] (Ai); mu = 1 without Ai.
  R mu = 1;
  if (ai) {
    R dev = 0;
    for (int j = 0; j < 6; ++j) dev = dev + r_abs<R>(g[j]);
    mu = dev / R(6) + mu0;
  }
  o->mu = mu;
  // eqs. (19)-(21) with L = 1, q = 1 (fixed after Table 1).
  const R beta_k[4] = {b0, b1, b2, b3};
  R alpha[4], asum = 0;
  for (int k = 0; k < 4; ++k) {
    R gamma_k = r_pow<R>(tau / (beta_k[k] + eps * mu * mu), p);
    alpha[k] = (R(D_NUM[k]) / R(D_DEN)) * (R(1) + gamma_k);
  }
  for (int k = 0; k < 4; ++k) asum = asum + alpha[sum_ix(k, 4)];
  // eq. (14): convex combination of the candidate fluxes.
  R fh = 0;
  for (int k = 0; k < 4; ++k) o->omega[k] = alpha[k] / asum;
  for (int k = 0; k < 4; ++k) fh = fh + o->omega[sum_ix(k, 4)] * o->fk[sum_ix(k, 4)];
  o->fhat = fh;
}

double za6(const double f[6], double eps, double mu0, double p, int ai) {
  ZA6Out<double> o;
  za6_flux<double>(f, eps, mu0, p, ai, &o);
  return o.fhat;
}

// ---------------------------------------------------------------------------
// Appendix: the fourth-, eighth- and tenth-order schemes (r = 2, 4, 5), with
// the coefficient tables as printed there; the sixth-order tables of
// Section 3 give r = 3.  Rows written "rev(.)" in the paper are reversed here.
// ---------------------------------------------------------------------------
struct OrderTable {
  int r;
  std::vector<int> c2r;                         // eq. (10) analogue, / c2r_den
  int c2r_den;
  std::vector<std::vector<int>> ck;             // r + 1 rows of r, / ck_den
  int ck_den;
  std::vector<int> d;                           // r + 1, / d_den
  int d_den;
  std::vector<std::vector<std::vector<int>>> B;  // B_0 .. B_{r-1}, B_d (r x r), / b_den
  int b_den;
  std::vector<int> ctau;                        // 2r
};

std::vector<int> rev1(const std::vector<int> &v) { return std::vector<int>(v.rbegin(), v.rend()); }
std::vector<std::vector<int>> rev2(const std::vector<std::vector<int>> &M) {
  const int n = (int)M.size();
  std::vector<std::vector<int>> R(n, std::vector<int>(n));
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) R[a][b] = M[n - 1 - a][n - 1 - b];
  return R;
}

OrderTable make_table(int r) {
  OrderTable t;
  t.r = r;
  if (r == 2) {  // Appendix A.1
    t.c2r = {-1, 7, 7, -1};
    t.c2r_den = 12;
    std::vector<int> c0 = {-1, 3}, c1 = {1, 1};
    t.ck = {c0, c1, rev1(c0)};
    t.ck_den = 2;
    t.d = {1, 4, 1};
    t.d_den = 6;
    std::vector<std::vector<int>> B0 = {{1, -1}, {-1, 1}}, Bd = {{1, -1}, {-1, 1}};
    t.B = {B0, rev2(B0), Bd};
    t.b_den = 1;
    t.ctau = {-1, 3, -3, 1};
  } else if (r == 3) {  // Section 3
    t.c2r = {1, -8, 37, 37, -8, 1};
    t.c2r_den = 60;
    t.ck = {{2, -7, 11}, {-1, 5, 2}, {2, 5, -1}, {11, -7, 2}};
    t.ck_den = 6;
    t.d = {1, 9, 9, 1};
    t.d_den = 20;
    std::vector<std::vector<int>> B0 = {{8, -19, 11}, {-19, 50, -31}, {11, -31, 20}};
    std::vector<std::vector<int>> B1 = {{8, -13, 5}, {-13, 26, -13}, {5, -13, 8}};
    std::vector<std::vector<int>> Bd = {{44, -73, 29}, {-73, 122, -49}, {29, -49, 20}};
    t.B = {B0, B1, rev2(B0), Bd};
    t.b_den = 6;
    t.ctau = {-1, 5, -10, 10, -5, 1};
  } else if (r == 4) {  // Appendix A.2
    t.c2r = {-3, 29, -139, 533, 533, -139, 29, -3};
    t.c2r_den = 840;
    std::vector<int> c0 = {-3, 13, -23, 25}, c1 = {1, -5, 13, 3}, c2 = {-1, 7, 7, -1};
    t.ck = {c0, c1, c2, rev1(c1), rev1(c0)};
    t.ck_den = 12;
    t.d = {1, 16, 36, 16, 1};
    t.d_den = 70;
    std::vector<std::vector<int>> B0 = {{547, -1941, 2321, -927}, {-1941, 7043, -8623, 3521},
                                        {2321, -8623, 11003, -4701}, {-927, 3521, -4701, 2107}};
    std::vector<std::vector<int>> B1 = {{267, -821, 801, -247}, {-821, 2843, -2983, 961},
                                        {801, -2983, 3443, -1261}, {-247, 961, -1261, 547}};
    std::vector<std::vector<int>> Bd = {{7107, -16901, 13521, -3727}, {-16901, 40643, -32863, 9121},
                                        {13521, -32863, 26843, -7501}, {-3727, 9121, -7501, 2107}};
    t.B = {B0, B1, rev2(B1), rev2(B0), Bd};
    t.b_den = 240;
    t.ctau = {-1, 7, -21, 35, -35, 21, -7, 1};
  } else {  // r == 5, Appendix A.3
    t.c2r = {2, -23, 127, -473, 1627, 1627, -473, 127, -23, 2};
    t.c2r_den = 2520;
    std::vector<int> c0 = {12, -63, 137, -163, 137}, c1 = {-3, 17, -43, 77, 12},
                     c2 = {2, -13, 47, 27, -3};
    t.ck = {c0, c1, c2, rev1(c2), rev1(c1), rev1(c0)};
    t.ck_den = 60;
    t.d = {1, 25, 100, 100, 25, 1};
    t.d_den = 252;
    std::vector<std::vector<int>> B0 = {{45316, -208501, 364863, -288007, 86329},
                                        {-208501, 965926, -1704396, 1358458, -411487},
                                        {364863, -1704396, 3042786, -2462076, 758823},
                                        {-288007, 1358458, -2462076, 2041126, -649501},
                                        {86329, -411487, 758823, -649501, 215836}};
    std::vector<std::vector<int>> B1 = {{13816, -60871, 99213, -70237, 18079},
                                        {-60871, 277126, -464976, 337018, -88297},
                                        {99213, -464976, 812586, -611976, 165153},
                                        {-70237, 337018, -611976, 485446, -140251},
                                        {18079, -88297, 165153, -140251, 45316}};
    std::vector<std::vector<int>> B2 = {{13816, -51001, 67923, -38947, 8209},
                                        {-51001, 209926, -299076, 179098, -38947},
                                        {67923, -299076, 462306, -299076, 67923},
                                        {-38947, 179098, -299076, 209926, -51001},
                                        {8209, -38947, 67923, -51001, 13816}};
    std::vector<std::vector<int>> Bd = {{942016, -2964751, 3597813, -2004757, 429679},
                                        {-2964751, 9449926, -11584896, 6499258, -1399537},
                                        {3597813, -11584896, 14319786, -8079576, 1746873},
                                        {-2004757, 6499258, -8079576, 4577926, -992851},
                                        {429679, -1399537, 1746873, -992851, 215836}};
    t.B = {B0, B1, B2, rev2(B1), rev2(B0), Bd};
    t.b_den = 10080;
    t.ctau = {-1, 9, -36, 84, -126, 126, -84, 36, -9, 1};
  }
  return t;
}

const OrderTable &table_of(int r) {
  static const OrderTable t2 = make_table(2), t3 = make_table(3), t4 = make_table(4),
                          t5 = make_table(5);
  return r == 2 ? t2 : (r == 3 ? t3 : (r == 4 ? t4 : t5));
}

// Central-upwind WENO flux of order 2r at x_{i+1/2} from f[0 .. 2r-1] =
// f_{i-r+1} .. f_{i+r} (Section 2: eqs. (9)-(22) with the tables above; the
// downwind indicator is the mean of all r + 1 local ones, eq. (16)).  The
// indicators are evaluated on shifted data as in za6_flux.
double zar_flux(int r, const double *f, double eps, double mu0, double p, int ai) {
  const OrderTable &t = table_of(r);
  const int n = 2 * r;
  std::vector<double> fk(r + 1), beta(r + 1);
  for (int k = 0; k <= r; ++k) {  // candidate fluxes on S_k
    double s = 0;
    for (int m = 0; m < r; ++m) s += (double)t.ck[k][m] * f[k + m];
    fk[k] = s / t.ck_den;
  }
  double bsum = 0;
  for (int k = 0; k <= r; ++k) {  // beta_0 .. beta_{r-1} and beta_d (k = r)
    std::vector<double> g(r);
    for (int m = 0; m < r; ++m) g[m] = f[k + m] - f[k];
    double s = 0;
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) s += g[a] * (double)t.B[k][a][b] * g[b];
    s /= t.b_den;
    if (k < r) beta[k] = s;
    bsum += s;
  }
  beta[r] = bsum / (r + 1);  // eq. (16)
  double mean = 0;
  for (int j = 0; j < n; ++j) mean += f[j];
  mean /= n;
  double tr = 0;
  for (int j = 0; j < n; ++j) tr += (double)t.ctau[j] * (f[j] - mean);
  const double tau = tr * tr;  // eq. (17)
  double mu = 1;
  if (ai) {  // eq. (22)
    double dev = 0;
    for (int j = 0; j < n; ++j) dev += std::fabs(f[j] - mean);
    mu = dev / n + mu0;
  }
  double asum = 0;
  std::vector<double> al(r + 1);
  for (int k = 0; k <= r; ++k) {  // eqs. (19)-(21), L = q = 1
    const double G = r_pow<double>(tau / (beta[k] + eps * mu * mu), p);
    al[k] = ((double)t.d[k] / t.d_den) * (1.0 + G);
  }
  for (int k = 0; k <= r; ++k) asum += al[sum_ix(k, r + 1)];
  double fh = 0;
  for (int q = 0; q <= r; ++q) {  // eq. (14)
    const int k = sum_ix(q, r + 1);
    fh += (al[k] / asum) * fk[k];
  }
  return fh;
}

// ---------------------------------------------------------------------------
// Euler equations (Section 4.2, eq. (25); its 2D form for Section 4.3).
// State order: (rho, rho u, E) in 1D, (rho, rho u, rho v, E) in 2D.
// ---------------------------------------------------------------------------
struct Prim {
  double rho, u, v, p, H;
};

bool finite(double x) { return std::isfinite(x); }

// Primitive variables from one conserved state; false if nonphysical.
bool to_prim(int nc, const double *U, double gamma, Prim *w) {
  double rho = U[0];
  double u = U[1] / rho;
  double v = (nc == 4) ? U[2] / rho : 0.0;
  double E = U[nc - 1];
  double p = (gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  w->rho = rho;
  w->u = u;
  w->v = v;
  w->p = p;
  w->H = (E + p) / rho;
  return rho > 0 && p > 0 && finite(rho) && finite(p) && finite(u) && finite(v);
}

// Physical flux in direction dir (0 = x, 1 = y).
void euler_flux(int nc, int dir, const double *U, const Prim &w, double *F) {
  double E = U[nc - 1];
  if (nc == 3) {
    F[0] = w.rho * w.u;
    F[1] = w.rho * w.u * w.u + w.p;
    F[2] = (E + w.p) * w.u;
    return;
  }
  double un = (dir == 0) ? w.u : w.v;
  F[0] = w.rho * un;
  F[1] = w.rho * w.u * un + (dir == 0 ? w.p : 0.0);
  F[2] = w.rho * w.v * un + (dir == 1 ? w.p : 0.0);
  F[3] = (E + w.p) * un;
}

// Eigenvalues of the flux Jacobian at one state, in the order of the
// right-eigenvector columns built below.
void euler_eigs(int nc, int dir, const Prim &w, double gamma, double *lam) {
  double c = std::sqrt(gamma * w.p / w.rho);
  double un = (dir == 0) ? w.u : w.v;
  if (nc == 3) {
    lam[0] = un - c;
    lam[1] = un;
    lam[2] = un + c;
  } else {
    lam[0] = un - c;
    lam[1] = un;
    lam[2] = un;
    lam[3] = un + c;
  }
}

// Right eigenvectors of the Euler flux Jacobian at the state (u, v, H, c), as
// columns R[row][col] (textbook gas dynamics; the paper uses the
// characteristic-wise splitting of its reference [ShuSpringer], Section 4.2).
void right_eigvecs(int nc, int dir, double u, double v, double H, double c, double R[4][4]) {
  std::memset(R, 0, sizeof(double) * 16);
  if (nc == 3) {
    double cols[3][3] = {{1.0, u - c, H - u * c}, {1.0, u, 0.5 * u * u}, {1.0, u + c, H + u * c}};
    for (int k = 0; k < 3; ++k)
      for (int r = 0; r < 3; ++r) R[r][k] = cols[k][r];
    return;
  }
  double q2 = u * u + v * v;
  if (dir == 0) {
    double cols[4][4] = {{1.0, u - c, v, H - u * c},
                         {1.0, u, v, 0.5 * q2},
                         {0.0, 0.0, 1.0, v},
                         {1.0, u + c, v, H + u * c}};
    for (int k = 0; k < 4; ++k)
      for (int r = 0; r < 4; ++r) R[r][k] = cols[k][r];
  } else {
    double cols[4][4] = {{1.0, u, v - c, H - v * c},
                         {1.0, u, v, 0.5 * q2},
                         {0.0, 1.0, 0.0, u},
                         {1.0, u, v + c, H + v * c}};
    for (int k = 0; k < 4; ++k)
      for (int r = 0; r < 4; ++r) R[r][k] = cols[k][r];
  }
}

// Inverse of an n x n matrix by Gauss-Jordan elimination with partial
// pivoting (plain linear algebra; gives the left eigenvectors L = R^{-1}).
bool invert(int n, const double A_in[4][4], double Ainv[4][4]) {
  double A[4][8];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) A[r][c] = (c < n) ? A_in[r][c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (A[piv][col] == 0.0) return false;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) std::swap(A[piv][c], A[col][c]);
    double d = A[col][col];
    for (int c = 0; c < 2 * n; ++c) A[col][c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = A[r][col];
      for (int c = 0; c < 2 * n; ++c) A[r][c] -= f * A[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r][c] = A[r][c + n];
  return true;
}

int ncomp_of(const ora_grid *g) {
  if (g->system != 1) return 1;
  return g->ndim == 1 ? 3 : 4;
}

// Scalar fluxes of Section 4.1: linear advection f = a u; Burgers f = u^2/2
// (convex); Buckley-Leverett f = u^2 / (u^2 + 0.25 (1-u)^2) (nonconvex,
// Table 5).  f' is their derivative.
double scalar_flux(const ora_grid *g, double u) {
  if (g->system == 2) return 0.5 * u * u;
  if (g->system == 3) return u * u / (u * u + 0.25 * (1.0 - u) * (1.0 - u));
  return g->adv_speed * u;
}

double scalar_dflux(const ora_grid *g, double u) {
  if (g->system == 2) return u;
  if (g->system == 3) {
    const double D = u * u + 0.25 * (1.0 - u) * (1.0 - u);
    return 0.5 * u * (1.0 - u) / (D * D);
  }
  return g->adv_speed;
}

// Maximiser of the Buckley-Leverett f' on [0, 1] (f' >= 0 there, zero at both
// ends and unimodal), by golden-section search.
double bl_speed_argmax() {
  ora_grid g;
  std::memset(&g, 0, sizeof(g));
  g.system = 3;
  const double r = 0.5 * (std::sqrt(5.0) - 1.0);
  double a = 0.0, b = 1.0;
  for (int it = 0; it < 200 && b - a > 1e-15; ++it) {
    const double c = b - r * (b - a), d = a + r * (b - a);
    if (scalar_dflux(&g, c) > scalar_dflux(&g, d))
      b = d;
    else
      a = c;
  }
  return 0.5 * (a + b);
}

// Eq. (6) for a scalar flux: alpha = max |f'(Q)| over the states Q between the
// smallest and largest value of the data (reading: for a nonconvex flux the
// largest speed of a Riemann fan lies inside that range, not at a cell state;
// for a convex or linear flux this is the maximum over the cells).
double scalar_alpha(const ora_grid *g, double umin, double umax) {
  double a = std::fmax(std::fabs(scalar_dflux(g, umin)), std::fabs(scalar_dflux(g, umax)));
  if (g->system == 3) {
    const double us = bl_speed_argmax();
    if (umin <= us && us <= umax) a = std::fmax(a, std::fabs(scalar_dflux(g, us)));
  }
  return a;
}

// Ghost-cell index map (3 ghosts per side for the 6-point stencil):
// transmissive = zero-order extrapolation (index clamp), periodic = wrap.
int64_t ghost(int64_t k, int64_t n, int bc) {
  if (bc == 1) return ((k % n) + n) % n;
  if (k < 0) return 0;
  if (k >= n) return n - 1;
  return k;
}

// Numerical flux at the face between stencil cells 2 and 3 of st[6][nc]
// (cells i-2 .. i+3 along direction dir).  alpha[nc] are the GLF speeds.
// Scalar advection: f(u) = a u, alpha = |a| (eq. (6)).
// Euler: characteristic-wise Lax-Friedrichs splitting (Section 4.2): the face
// state is the Roe average of cells i and i+1; every stencil state and its
// flux are projected on the left eigenvectors, split by eq. (6) field by
// field, reconstructed by WENO-ZA6 (positive flux on the stencil, negative
// flux on its mirror image) and projected back with the right eigenvectors.
int order_r(const ora_grid *g) {
  const int o = g->order == 0 ? 6 : g->order;
  return o / 2;
}

// One WENO flux of the grid's order from n = 2r values.
double weno_flux(const ora_grid *g, const double *f) {
  const int r = order_r(g);
  if (r == 3) return za6(f, g->eps, g->mu0, g->p, g->ai);
  return zar_flux(r, f, g->eps, g->mu0, g->p, g->ai);
}

// Roe-averaged state of two neighbouring cells and the eigen-system of the
// flux Jacobian there (the face state of the characteristic-wise splitting,
// Section 4.2): u, v and H averaged with the weights sqrt(rho_L), sqrt(rho_R),
// c^2 = (gamma - 1)(H - q^2/2), R from right_eigvecs, L = R^{-1} by
// Gauss-Jordan, and the eigenvalues lam in the order of R's columns.
struct RoeSys {
  double u, v, H, c;
  double R[4][4], L[4][4], lam[4];
};

bool roe_system(int nc, int dir, double gamma, const Prim &wl, const Prim &wr, RoeSys *o) {
  double sl = std::sqrt(wl.rho), sr = std::sqrt(wr.rho);
  double u = (sl * wl.u + sr * wr.u) / (sl + sr);
  double v = (sl * wl.v + sr * wr.v) / (sl + sr);
  double H = (sl * wl.H + sr * wr.H) / (sl + sr);
  double c2 = (gamma - 1.0) * (H - 0.5 * (u * u + v * v));
  if (!(c2 > 0) || !finite(c2)) return false;
  double c = std::sqrt(c2);
  o->u = u;
  o->v = v;
  o->H = H;
  o->c = c;
  right_eigvecs(nc, dir, u, v, H, c, o->R);
  std::memset(o->L, 0, sizeof(o->L));
  if (!invert(nc, o->R, o->L)) return false;
  const double un = (dir == 0) ? u : v;
  for (int k = 0; k < 4; ++k) o->lam[k] = 0.0;
  if (nc == 3) {
    o->lam[0] = un - c;
    o->lam[1] = un;
    o->lam[2] = un + c;
  } else {
    o->lam[0] = un - c;
    o->lam[1] = un;
    o->lam[2] = un;
    o->lam[3] = un + c;
  }
  return true;
}

int face_flux(const ora_grid *g, int dir, const double st[10][4], const double *alpha,
              double *Fhat) {
  const int nc = ncomp_of(g);
  const int r = order_r(g), n = 2 * r;
  if (g->system != 1) {
    double fp[10], fm[10];
    for (int j = 0; j < n; ++j) {
      double f = scalar_flux(g, st[j][0]);
      fp[j] = 0.5 * (f + alpha[0] * st[j][0]);
      fm[n - 1 - j] = 0.5 * (f - alpha[0] * st[j][0]);
    }
    Fhat[0] = weno_flux(g, fp) + weno_flux(g, fm);
    return 0;
  }
  Prim w[10];
  double F[10][4];
  for (int j = 0; j < n; ++j) {
    if (!to_prim(nc, st[j], g->gamma, &w[j])) return 2;
    euler_flux(nc, dir, st[j], w[j], F[j]);
  }
  // Roe average of cells i (stencil index r-1) and i+1 (index r), and its
  // eigen-system.
  RoeSys rs;
  if (!roe_system(nc, dir, g->gamma, w[r - 1], w[r], &rs)) return 2;
  const double(&R)[4][4] = rs.R;
  const double(&L)[4][4] = rs.L;
  double h[4];
  for (int m = 0; m < nc; ++m) {
    double fp[10], fm[10];
    for (int j = 0; j < n; ++j) {
      double wc = 0, gc = 0;
      for (int q = 0; q < nc; ++q) {
        const int k = sum_ix(q, nc);
        wc += L[m][k] * st[j][k];
        gc += L[m][k] * F[j][k];
      }
      fp[j] = 0.5 * (gc + alpha[m] * wc);          // f^+ of eq. (6)
      fm[n - 1 - j] = 0.5 * (gc - alpha[m] * wc);  // f^- of eq. (6), mirrored
    }
    h[m] = weno_flux(g, fp) + weno_flux(g, fm);
  }
  for (int rr = 0; rr < nc; ++rr) {
    double sum = 0;
    for (int q = 0; q < nc; ++q) sum += R[rr][sum_ix(q, nc)] * h[sum_ix(q, nc)];
    Fhat[rr] = sum;
  }
  return 0;
}

// Load the 2r-cell stencil of face (i+1/2) along x in row j (cells i-r+1 ..
// i+r), or of face (j+1/2) along y in column i, of problem b.
void load_stencil(const ora_grid *g, const double *U, int64_t b, int dir, int64_t j, int64_t i,
                  double st[10][4]) {
  const int nc = ncomp_of(g);
  const int r = order_r(g);
  const int64_t nx = g->nx, ny = g->ny;
  const double *Ub = U + b * nc * nx * ny;
  for (int s = 0; s < 2 * r; ++s) {
    int64_t ii = i, jj = j;
    if (dir == 0)
      ii = ghost(i - r + 1 + s, nx, g->bc_x);
    else
      jj = ghost(j - r + 1 + s, ny, g->bc_y);
    for (int k = 0; k < nc; ++k) st[s][k] = Ub[(k * ny + jj) * nx + ii];
  }
}

int check_grid(const ora_grid *g) {
  if (!g || g->nbatch < 1 || g->nx < 1 || g->ny < 1) return 1;
  if (g->ndim != 1 && g->ndim != 2) return 1;
  if (g->ndim == 1 && g->ny != 1) return 1;
  if (g->system < 0 || g->system > 3) return 1;
  if (g->order != 0 && g->order != 4 && g->order != 6 && g->order != 8 && g->order != 10) return 1;
  if (g->system != 1 && g->ndim != 1) return 1;
  return 0;
}

// One cell's L(U): faces i-1/2, i+1/2 (and j-1/2, j+1/2 in 2D), eq. (5).
int rhs_cell(const ora_grid *g, const double *U, const double *alpha, int64_t b, int64_t j,
             int64_t i, double *out) {
  const int nc = ncomp_of(g);
  double st[10][4], Fl[4], Fr[4];
  const double *al = alpha + b * 8;
  load_stencil(g, U, b, 0, j, i - 1, st);
  int e = face_flux(g, 0, st, al, Fl);
  if (e) return e;
  load_stencil(g, U, b, 0, j, i, st);
  e = face_flux(g, 0, st, al, Fr);
  if (e) return e;
  for (int k = 0; k < nc; ++k) out[k] = -(Fr[k] - Fl[k]) / g->dx;
  if (g->ndim == 2) {
    double Gl[4], Gr[4];
    load_stencil(g, U, b, 1, j - 1, i, st);
    e = face_flux(g, 1, st, al + 4, Gl);
    if (e) return e;
    load_stencil(g, U, b, 1, j, i, st);
    e = face_flux(g, 1, st, al + 4, Gr);
    if (e) return e;
    for (int k = 0; k < nc; ++k) out[k] = out[k] - (Gr[k] - Gl[k]) / g->dy;
  }
  return 0;
}

// Section 3.1, eq. (26) test function and Tables 3-4.  Reading (checked
// against every printed entry): the nodes are x_j = -1 + j dx including both
// end points, f is evaluated analytically beyond [-1, 1], only the positive
// flux is reconstructed (the advection speed is positive), mu = 1.
template <class R>
double operator_error_t(int ncp, int inv_dx, double p, int eps_variable) {
  const int n = 2 * inv_dx;  // intervals on [-1, 1]
  const R dx = R(1) / R(inv_dx);
  R eps = eps_variable ? R(1) : R(1e-40);
  if (eps_variable)
    for (int k = 0; k < 2 * (ncp - 1); ++k) eps = eps * dx;  // dx^(2(ncp-1))
  auto fun = [&](R x) {
    R xp = 1;
    for (int k = 0; k < ncp + 1; ++k) xp = xp * x;
    return xp * r_exp<R>(R(0.75) * x);
  };
  auto dfun = [&](R x) {
    R xp = 1;  // x^ncp
    for (int k = 0; k < ncp; ++k) xp = xp * x;
    R e = r_exp<R>(R(0.75) * x);
    return R(ncp + 1) * xp * e + R(0.75) * xp * x * e;
  };
  // f_hat_{j+1/2} for j = -1 .. n.
  std::vector<R> fh(n + 2);
  for (int j = -1; j <= n; ++j) {
    R f[6];
    for (int s = 0; s < 6; ++s) f[s] = fun(R(-1) + R(j - 2 + s) * dx);
    ZA6Out<R> o;
    za6_flux<R>(f, eps, R(1e-40), p, 0, &o);
    fh[j + 1] = o.fhat;
  }
  R emax = 0;
  for (int j = 0; j <= n; ++j) {
    R d = (fh[j + 1] - fh[j]) / dx - dfun(R(-1) + R(j) * dx);
    if (r_abs<R>(d) > emax) emax = r_abs<R>(d);
  }
  return (double)emax;
}

}  // namespace

// ===========================================================================
// Exported functions.
// ===========================================================================
extern "C" {

double ora_za6_flux(const double f[6], double eps, double mu0, double p, int ai, double *detail) {
  ZA6Out<double> o;
  za6_flux<double>(f, eps, mu0, p, ai, &o);
  if (detail) {
    for (int k = 0; k < 4; ++k) detail[k] = o.fk[k];
    for (int k = 0; k < 5; ++k) detail[4 + k] = o.beta[k];
    detail[9] = o.tau;
    detail[10] = o.mu;
    for (int k = 0; k < 4; ++k) detail[11 + k] = o.omega[k];
    detail[15] = o.fhat;
  }
  return o.fhat;
}

double ora_za6_flux_quad(const double f[6], double eps, double mu0, double p, int ai) {
  quad fq[6];
  for (int j = 0; j < 6; ++j) fq[j] = (quad)f[j];
  ZA6Out<quad> o;
  za6_flux<quad>(fq, (quad)eps, (quad)mu0, p, ai, &o);
  return (double)o.fhat;
}

double ora_za_flux(int order, const double *f, double eps, double mu0, double p, int ai) {
  const int r = order / 2;
  if (r < 2 || r > 5 || 2 * r != order) return NAN;
  return zar_flux(r, f, eps, mu0, p, ai);
}

int ora_coefficients_r(int order, double *out) {
  const int r = order / 2;
  if (r < 2 || r > 5 || 2 * r != order) return 1;
  const OrderTable &t = table_of(r);
  int n = 0;
  for (int j = 0; j < 2 * r; ++j) out[n++] = (double)t.c2r[j] / t.c2r_den;
  for (int k = 0; k <= r; ++k)
    for (int m = 0; m < r; ++m) out[n++] = (double)t.ck[k][m] / t.ck_den;
  for (int k = 0; k <= r; ++k) out[n++] = (double)t.d[k] / t.d_den;
  for (int k = 0; k <= r; ++k)
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) out[n++] = (double)t.B[k][a][b] / t.b_den;
  for (int j = 0; j < 2 * r; ++j) out[n++] = (double)t.ctau[j];
  return 0;
}

void ora_coefficients(double *out) {
  int n = 0;
  for (int j = 0; j < 6; ++j) out[n++] = (double)C6_NUM[j] / C6_DEN;
  for (int k = 0; k < 4; ++k)
    for (int m = 0; m < 3; ++m) out[n++] = (double)CK_NUM[k][m] / CK_DEN;
  for (int k = 0; k < 4; ++k) out[n++] = (double)D_NUM[k] / D_DEN;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[n++] = (double)B0_NUM[a][b] / B_DEN;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[n++] = (double)B1_NUM[a][b] / B_DEN;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[n++] = (double)b2_num(a, b) / B_DEN;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[n++] = (double)BD_NUM[a][b] / B_DEN;
  for (int j = 0; j < 6; ++j) out[n++] = (double)CTAU[j];
}

double ora_operator_error(int ncp, int inv_dx, double p, int eps_variable, int use_quad) {
  if (ncp < 0 || inv_dx < 3) return -1.0;
  if (use_quad) return operator_error_t<quad>(ncp, inv_dx, p, eps_variable);
  return operator_error_t<double>(ncp, inv_dx, p, eps_variable);
}

int ora_roe_face(int nc, int dir, double gamma, const double *UL, const double *UR,
                 double *out) {
  if ((nc != 3 && nc != 4) || dir < 0 || dir > (nc == 4 ? 1 : 0) || !(gamma > 1.0)) return 1;
  Prim wl, wr;
  if (!to_prim(nc, UL, gamma, &wl) || !to_prim(nc, UR, gamma, &wr)) return 2;
  RoeSys rs;
  if (!roe_system(nc, dir, gamma, wl, wr, &rs)) return 2;
  out[0] = rs.u;
  out[1] = rs.v;
  out[2] = rs.H;
  out[3] = rs.c;
  for (int r = 0; r < 4; ++r)
    for (int k = 0; k < 4; ++k) {
      out[4 + 4 * r + k] = rs.R[r][k];
      out[20 + 4 * r + k] = rs.L[r][k];
    }
  for (int k = 0; k < 4; ++k) out[36 + k] = rs.lam[k];
  return 0;
}

// Eq. (6): alpha = max |f'(Q)|.  Reading: the maximum is taken over all cells
// of the stage input, per problem, per direction and per characteristic field
// (alpha_mode 0) or once over all fields (alpha_mode 1).
int ora_alpha(const ora_grid *g, const double *U, double *alpha) {
  if (check_grid(g)) return 1;
  const int nc = ncomp_of(g);
  const int64_t nx = g->nx, ny = g->ny, plane = nx * ny;
  for (int64_t b = 0; b < g->nbatch; ++b) {
    double *al = alpha + b * 8;
    for (int k = 0; k < 8; ++k) al[k] = 0.0;
    if (g->system == 0) {
      al[0] = std::fabs(g->adv_speed);
      continue;
    }
    const double *Ub = U + b * nc * plane;
    if (g->system != 1) {
      double umin = Ub[0], umax = Ub[0];
      for (int64_t c = 0; c < plane; ++c) {
        if (!std::isfinite(Ub[c])) return 2;
        umin = std::fmin(umin, Ub[c]);
        umax = std::fmax(umax, Ub[c]);
      }
      al[0] = scalar_alpha(g, umin, umax);
      continue;
    }
    for (int64_t c = 0; c < plane; ++c) {
      double s[4];
      for (int k = 0; k < nc; ++k) s[k] = Ub[k * plane + c];
      Prim w;
      if (!to_prim(nc, s, g->gamma, &w)) return 2;
      for (int dir = 0; dir < g->ndim; ++dir) {
        double lam[4];
        euler_eigs(nc, dir, w, g->gamma, lam);
        for (int m = 0; m < nc; ++m)
          if (std::fabs(lam[m]) > al[dir * 4 + m]) al[dir * 4 + m] = std::fabs(lam[m]);
      }
    }
    if (g->alpha_mode == 1) {
      for (int dir = 0; dir < 2; ++dir) {
        double a = 0;
        for (int m = 0; m < nc; ++m) a = std::fmax(a, al[dir * 4 + m]);
        for (int m = 0; m < nc; ++m) al[dir * 4 + m] = (dir < g->ndim) ? a : 0.0;
      }
    }
  }
  return 0;
}

int ora_rhs(const ora_grid *g, const double *U, const double *alpha, double *L) {
  if (check_grid(g)) return 1;
  const int nc = ncomp_of(g);
  const int64_t nx = g->nx, ny = g->ny, plane = nx * ny;
  std::vector<double> Fx((size_t)(nx + 1) * 4), Gy((size_t)(ny + 1) * 4);
  for (int64_t b = 0; b < g->nbatch; ++b) {
    const double *al = alpha + b * 8;
    double *Lb = L + b * nc * plane;
    // x sweep: faces i+1/2 for i = -1 .. nx-1 of every row.
    for (int64_t j = 0; j < ny; ++j) {
      for (int64_t i = -1; i < nx; ++i) {
        double st[10][4];
        load_stencil(g, U, b, 0, j, i, st);
        int e = face_flux(g, 0, st, al, &Fx[(size_t)(i + 1) * 4]);
        if (e) return e;
      }
      for (int64_t i = 0; i < nx; ++i)
        for (int k = 0; k < nc; ++k)
          Lb[(k * ny + j) * nx + i] = -(Fx[(size_t)(i + 1) * 4 + k] - Fx[(size_t)i * 4 + k]) / g->dx;
    }
    if (g->ndim == 1) continue;
    // y sweep: faces j+1/2 for j = -1 .. ny-1 of every column.
    for (int64_t i = 0; i < nx; ++i) {
      for (int64_t j = -1; j < ny; ++j) {
        double st[10][4];
        load_stencil(g, U, b, 1, j, i, st);
        int e = face_flux(g, 1, st, al + 4, &Gy[(size_t)(j + 1) * 4]);
        if (e) return e;
      }
      for (int64_t j = 0; j < ny; ++j)
        for (int k = 0; k < nc; ++k)
          Lb[(k * ny + j) * nx + i] =
              Lb[(k * ny + j) * nx + i] - (Gy[(size_t)(j + 1) * 4 + k] - Gy[(size_t)j * 4 + k]) / g->dy;
    }
  }
  return 0;
}

int ora_rhs_cell(const ora_grid *g, const double *U, const double *alpha, int64_t b, int64_t j,
                 int64_t i, double *out) {
  if (check_grid(g)) return 1;
  if (b < 0 || b >= g->nbatch || j < 0 || j >= g->ny || i < 0 || i >= g->nx) return 1;
  return rhs_cell(g, U, alpha, b, j, i, out);
}

// Reading of the silent CFL rule: 1D dt = cfl dx / max(|u| + c);
// 2D dt = cfl / (max(|u| + c)/dx + max(|v| + c)/dy), from the step's input.
int ora_cfl_dt(const ora_grid *g, const double *U, double cfl, double *dt) {
  if (check_grid(g)) return 1;
  const int nc = ncomp_of(g);
  const int64_t plane = g->nx * g->ny;
  for (int64_t b = 0; b < g->nbatch; ++b) {
    if (g->system == 0) {
      dt[b] = cfl * g->dx / std::fabs(g->adv_speed);
      continue;
    }
    const double *Ub = U + b * nc * plane;
    if (g->system != 1) {
      double umin = Ub[0], umax = Ub[0];
      for (int64_t c = 0; c < plane; ++c) {
        umin = std::fmin(umin, Ub[c]);
        umax = std::fmax(umax, Ub[c]);
      }
      dt[b] = cfl * g->dx / scalar_alpha(g, umin, umax);
      continue;
    }
    double sx = 0, sy = 0;
    for (int64_t c = 0; c < plane; ++c) {
      double s[4];
      for (int k = 0; k < nc; ++k) s[k] = Ub[k * plane + c];
      Prim w;
      if (!to_prim(nc, s, g->gamma, &w)) return 2;
      double cs = std::sqrt(g->gamma * w.p / w.rho);
      sx = std::fmax(sx, std::fabs(w.u) + cs);
      sy = std::fmax(sy, std::fabs(w.v) + cs);
    }
    if (g->ndim == 1)
      dt[b] = cfl * g->dx / sx;
    else
      dt[b] = cfl / (sx / g->dx + sy / g->dy);
  }
  return 0;
}

// Third-order TVD (SSP) Runge-Kutta of Shu and Osher (Section 4 preamble):
//   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));
//   U^{n+1} = 1/3 U + 2/3 (U2 + dt L(U2)).
// The GLF speeds are recomputed from each stage's input.
int ora_ssprk3_step(const ora_grid *g, double *U, const double *dt) {
  if (check_grid(g)) return 1;
  const int nc = ncomp_of(g);
  const int64_t per = nc * g->nx * g->ny, tot = per * g->nbatch;
  std::vector<double> U1(tot), U2(tot), L(tot), al(g->nbatch * 8);
  int e = ora_alpha(g, U, al.data());
  if (e) return e;
  e = ora_rhs(g, U, al.data(), L.data());
  if (e) return e;
  for (int64_t b = 0; b < g->nbatch; ++b) {
    double h = dt[b] > 0 ? dt[b] : 0.0;
    for (int64_t q = b * per; q < (b + 1) * per; ++q) U1[q] = U[q] + h * L[q];
  }
  e = ora_alpha(g, U1.data(), al.data());
  if (e) return e;
  e = ora_rhs(g, U1.data(), al.data(), L.data());
  if (e) return e;
  for (int64_t b = 0; b < g->nbatch; ++b) {
    double h = dt[b] > 0 ? dt[b] : 0.0;
    for (int64_t q = b * per; q < (b + 1) * per; ++q)
      U2[q] = 0.75 * U[q] + 0.25 * (U1[q] + h * L[q]);
  }
  e = ora_alpha(g, U2.data(), al.data());
  if (e) return e;
  e = ora_rhs(g, U2.data(), al.data(), L.data());
  if (e) return e;
  for (int64_t b = 0; b < g->nbatch; ++b) {
    if (!(dt[b] > 0)) continue;
    double h = dt[b];
    for (int64_t q = b * per; q < (b + 1) * per; ++q)
      U[q] = (1.0 / 3.0) * U[q] + (2.0 / 3.0) * (U2[q] + h * L[q]);
  }
  return 0;
}

int ora_solve(const ora_grid *g, double *U, double cfl, double t0, double t_final,
              int64_t max_steps, double *t_out, int64_t *steps_out) {
  if (check_grid(g)) return 1;
  const int64_t nb = g->nbatch;
  std::vector<double> t(nb, t0), dt(nb);
  std::vector<int64_t> steps(nb, 0);
  std::vector<char> done(nb, 0);
  int status = 0;
  for (int64_t n = 0;; ++n) {
    bool all = true;
    for (int64_t b = 0; b < nb; ++b)
      if (!(t[b] < t_final)) done[b] = 1;
      else all = false;
    if (all) break;
    if (n >= max_steps) {
      status = 3;
      break;
    }
    int e = ora_cfl_dt(g, U, cfl, dt.data());
    if (e) {
      status = e;
      break;
    }
    std::vector<char> last(nb, 0);
    for (int64_t b = 0; b < nb; ++b) {
      if (done[b]) {
        dt[b] = 0.0;
        continue;
      }
      if (dt[b] >= t_final - t[b]) {  // clip the last step onto t_final
        dt[b] = t_final - t[b];
        last[b] = 1;
      }
    }
    e = ora_ssprk3_step(g, U, dt.data());
    if (e) {
      status = e;
      break;
    }
    for (int64_t b = 0; b < nb; ++b) {
      if (done[b]) continue;
      t[b] = last[b] ? t_final : t[b] + dt[b];
      steps[b] += 1;
    }
  }
  for (int64_t b = 0; b < nb; ++b) {
    if (t_out) t_out[b] = t[b];
    if (steps_out) steps_out[b] = steps[b];
  }
  return status;
}

// ---------------------------------------------------------------------------
// Exact Riemann solver for the 1D Euler equations (ideal gas), written from
// the standard wave-curve analysis of gas dynamics (e.g. E. F. Toro, "Riemann
// Solvers and Numerical Methods for Fluid Dynamics", ch. 4): the star
// pressure is the root of f_L(p) + f_R(p) + u_R - u_L = 0 with shock
// (Rankine-Hugoniot) or rarefaction (isentropic) branches; the root is found
// by bisection, which needs only that f is increasing in p.
// ---------------------------------------------------------------------------
static double wave_f(double p, double rk, double pk, double ck, double gamma) {
  if (p > pk) {
    double A = 2.0 / ((gamma + 1.0) * rk), B = (gamma - 1.0) / (gamma + 1.0) * pk;
    return (p - pk) * std::sqrt(A / (p + B));
  }
  return 2.0 * ck / (gamma - 1.0) * (std::pow(p / pk, (gamma - 1.0) / (2.0 * gamma)) - 1.0);
}

int ora_riemann_exact(double rl, double ul, double pl, double rr, double ur, double pr,
                      double gamma, double x0, double t, int64_t n, const double *x, double *rho,
                      double *u, double *p, double *star) {
  if (!(rl > 0 && rr > 0 && pl > 0 && pr > 0 && t > 0)) return 1;
  const double cl = std::sqrt(gamma * pl / rl), cr = std::sqrt(gamma * pr / rr);
  if (2.0 * (cl + cr) / (gamma - 1.0) <= ur - ul) return 2;  // vacuum
  auto F = [&](double ps) {
    return wave_f(ps, rl, pl, cl, gamma) + wave_f(ps, rr, pr, cr, gamma) + ur - ul;
  };
  double lo = 0.0, hi = std::fmax(pl, pr);
  while (F(hi) < 0) hi *= 2.0;
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (F(mid) < 0)
      lo = mid;
    else
      hi = mid;
  }
  const double ps = 0.5 * (lo + hi);
  const double us = 0.5 * (ul + ur) + 0.5 * (wave_f(ps, rr, pr, cr, gamma) - wave_f(ps, rl, pl, cl, gamma));
  if (star) {
    star[0] = ps;
    star[1] = us;
  }
  const double g1 = (gamma - 1.0) / (2.0 * gamma), g2 = (gamma + 1.0) / (2.0 * gamma);
  const double g6 = (gamma - 1.0) / (gamma + 1.0), g5 = 2.0 / (gamma + 1.0);
  for (int64_t k = 0; k < n; ++k) {
    const double S = (x[k] - x0) / t;
    double r, v, q;
    if (S <= us) {  // left of the contact
      if (ps > pl) {  // left shock
        double sl = ul - cl * std::sqrt(g2 * ps / pl + g1);
        if (S <= sl) {
          r = rl; v = ul; q = pl;
        } else {
          r = rl * (ps / pl + g6) / (g6 * ps / pl + 1.0); v = us; q = ps;
        }
      } else {  // left rarefaction
        double shl = ul - cl, cml = cl * std::pow(ps / pl, g1), stl = us - cml;
        if (S <= shl) {
          r = rl; v = ul; q = pl;
        } else if (S >= stl) {
          r = rl * std::pow(ps / pl, 1.0 / gamma); v = us; q = ps;
        } else {
          double base = g5 + g6 / cl * (ul - S);
          r = rl * std::pow(base, 2.0 / (gamma - 1.0));
          v = g5 * (cl + 0.5 * (gamma - 1.0) * ul + S);
          q = pl * std::pow(base, 2.0 * gamma / (gamma - 1.0));
        }
      }
    } else {  // right of the contact
      if (ps > pr) {  // right shock
        double sr = ur + cr * std::sqrt(g2 * ps / pr + g1);
        if (S >= sr) {
          r = rr; v = ur; q = pr;
        } else {
          r = rr * (ps / pr + g6) / (g6 * ps / pr + 1.0); v = us; q = ps;
        }
      } else {  // right rarefaction
        double shr = ur + cr, cmr = cr * std::pow(ps / pr, g1), str = us + cmr;
        if (S >= shr) {
          r = rr; v = ur; q = pr;
        } else if (S <= str) {
          r = rr * std::pow(ps / pr, 1.0 / gamma); v = us; q = ps;
        } else {
          double base = g5 - g6 / cr * (ur - S);
          r = rr * std::pow(base, 2.0 / (gamma - 1.0));
          v = g5 * (-cr + 0.5 * (gamma - 1.0) * ur + S);
          q = pr * std::pow(base, 2.0 * gamma / (gamma - 1.0));
        }
      }
    }
    rho[k] = r;
    u[k] = v;
    p[k] = q;
  }
  return 0;
}

}  // extern "C"
