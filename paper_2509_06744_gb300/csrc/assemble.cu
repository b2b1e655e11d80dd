// PUM assembly on the device (Section 4; Nitsche forms of Examples 5.1 and 5.4).
//
// The cover, the partition of unity and the local Legendre spaces are tensor products,
// so every integral of a_n and l_n factorises: a domain integral of a product of two
// derivatives of basis functions phi_i theta_i^k = X_i(x) Y_i(y) is the product of two
// 1-D integrals, a boundary integral is a 1-D integral times point values.  The host
// builds the small 1-D tables (Gauss-Legendre on the sub-intervals between partition-of-
// unity breakpoints, where every integrand is a polynomial); the device forms each d x d
// block of A (and of the prolongation P) as sums of products of table entries.
#include <algorithm>
#include <cmath>
#include <map>

#include "pum_internal.cuh"

namespace pum {
namespace {

// ----------------------------------------------------------------------------- 1-D math

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_q (q <= 32).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.resize(q);
  w.resize(q);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int n = 2; n <= q; ++n) {
        const double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) { p0 = 1.0; p1 = z; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Monomial coefficients of the Legendre polynomial P_j by (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1}.
std::vector<double> legendre_coeffs(int j) {
  std::vector<double> a{1.0}, b{0.0, 1.0};
  if (j == 0) return a;
  for (int n = 1; n < j; ++n) {
    std::vector<double> c(n + 2, 0.0);
    for (int i = 0; i <= n; ++i) c[i + 1] += (2.0 * n + 1.0) * b[i] / (n + 1.0);
    for (int i = 0; i < (int)a.size(); ++i) c[i] -= n * a[i] / (n + 1.0);
    a = b;
    b = c;
  }
  return b;
}

std::vector<double> poly_der(std::vector<double> c, int r) {
  for (int k = 0; k < r; ++k) {
    if (c.size() <= 1) return {0.0};
    std::vector<double> d(c.size() - 1);
    for (size_t i = 1; i < c.size(); ++i) d[i - 1] = c[i] * (double)i;
    c = d;
  }
  return c;
}

double poly_eval(const std::vector<double>& c, double t) {
  double s = 0.0;
  for (int i = (int)c.size() - 1; i >= 0; --i) s = s * t + c[i];
  return s;
}

struct Level1D {
  int m;
  explicit Level1D(int m_) : m(m_) {}
  double lo(int a) const { return std::max((a - 0.25) / m, 0.0); }
  double hi(int a) const { return std::min((a + 1.25) / m, 1.0); }
  std::vector<double> breakpoints() const {
    std::vector<double> v{0.0, 1.0};
    for (int a = 0; a < m; ++a)
      for (double fr : {0.25, 0.75}) {
        const double x = (a + fr) / m;
        if (x > 0.0 && x < 1.0) v.push_back(x);
      }
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    return v;
  }
  bool covers(int a, double l, double h) const {
    const double mid = 0.5 * (l + h);
    return lo(a) < mid && mid < hi(a);
  }
};

// S(t) = 10 t^3 - 15 t^4 + 6 t^5 and its derivatives.
double smoothstep(double t, int r) {
  static const std::vector<double> S{0.0, 0.0, 0.0, 10.0, -15.0, 6.0};
  return poly_eval(poly_der(S, r), t);
}

// r-th derivative of the 1-D partition-of-unity function of patch a: 1 on the patch's
// own zone ((a+1/4)h, (a+3/4)h) (extended to the domain boundary on boundary patches),
// S-blends of width h/2 towards the neighbours, 0 elsewhere.
double pu(const Level1D& L, int a, double x, int r) {
  const int m = L.m;
  const double h = 1.0 / m;
  const double own_lo = a > 0 ? (a + 0.25) / m : 0.0;
  const double own_hi = a < m - 1 ? (a + 0.75) / m : 1.0;
  if (x >= own_lo && x <= own_hi) return r == 0 ? 1.0 : 0.0;
  if (a > 0) {
    const double lo = (a - 0.25) / m;
    if (x >= lo && x < own_lo) {
      const double t = std::min(std::max((x - lo) / (0.5 * h), 0.0), 1.0);
      return smoothstep(t, r) * std::pow(2.0 / h, r);
    }
  }
  if (a < m - 1) {
    const double lo = (a + 0.75) / m, hi = (a + 1.25) / m;
    if (x > own_hi && x <= hi) {
      const double t = std::min(std::max((x - lo) / (0.5 * h), 0.0), 1.0);
      const double v = smoothstep(t, r) * std::pow(2.0 / h, r);
      return r == 0 ? 1.0 - v : -v;
    }
  }
  return 0.0;
}

struct Basis1D {
  std::vector<std::vector<std::vector<double>>> der;  // der[j][r] = coefficients of P_j^(r)
  explicit Basis1D(int p, int rmax) {
    der.resize(p + 1);
    for (int j = 0; j <= p; ++j)
      for (int r = 0; r <= rmax; ++r) der[j].push_back(poly_der(legendre_coeffs(j), r));
  }
  // r-th derivative of P_j(xi(x)) on the box [lo, hi]
  double local(int j, double lo, double hi, double x, int r) const {
    const double w = hi - lo;
    return poly_eval(der[j][r], (2.0 * x - lo - hi) / w) * std::pow(2.0 / w, r);
  }
};

double binom(int n, int k) {
  double c = 1.0;
  for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
  return c;
}

// n-th derivative of X_{a,j}(x) = phi_a(x) P_j(xi_a(x)) (Leibniz).
double factor(const Level1D& L, const Basis1D& B, int a, int j, double x, int n) {
  double s = 0.0;
  for (int r = 0; r <= n; ++r) {
    const double ph = pu(L, a, x, r);
    if (ph != 0.0) s += binom(n, r) * ph * B.local(j, L.lo(a), L.hi(a), x, n - r);
  }
  return s;
}

// ----------------------------------------------------------------------------- operators

struct Mono { int ax, ay; double c; };
using Op = std::vector<Mono>;

Op op_I() { return {{0, 0, 1.0}}; }
Op op_lap() { return {{2, 0, 1.0}, {0, 2, 1.0}}; }
// tr(S H(w)) = S11 w_xx + 2 S12 w_xy + S22 w_yy (Example 5.2); the Laplacian when S = I.
struct Aniso {
  bool on = false;
  double s11 = 1.0, s12 = 0.0, s22 = 1.0;
};
Op op_lapS(const Aniso& S) {
  if (!S.on) return op_lap();
  Op r;
  if (S.s11 != 0.0) r.push_back({2, 0, S.s11});
  if (S.s12 != 0.0) r.push_back({1, 1, 2.0 * S.s12});
  if (S.s22 != 0.0) r.push_back({0, 2, S.s22});
  return r;
}
Op op_bilap() { return {{4, 0, 1.0}, {2, 2, 2.0}, {0, 4, 1.0}}; }
Op op_dx(const Op& o) { Op r; for (auto m : o) r.push_back({m.ax + 1, m.ay, m.c}); return r; }
Op op_dy(const Op& o) { Op r; for (auto m : o) r.push_back({m.ax, m.ay + 1, m.c}); return r; }
Op op_dn(const Op& o, double nx, double ny) {
  Op r;
  if (nx != 0.0) for (auto m : o) r.push_back({m.ax + 1, m.ay, nx * m.c});
  if (ny != 0.0) for (auto m : o) r.push_back({m.ax, m.ay + 1, ny * m.c});
  return r;
}

struct Pair { Op v, u; double c; };

// a_n(v, u) of Example 5.1 (order 4; Example 5.2 with S) and Example 5.4 (order 6): domain part.
std::vector<Pair> interior_pairs(int order, const Aniso& S) {
  if (order == 4) return {{op_lapS(S), op_lapS(S), 1.0}};
  return {{op_dx(op_lap()), op_dx(op_lap()), 1.0}, {op_dy(op_lap()), op_dy(op_lap()), 1.0}};
}

// Boundary part on an edge with outward normal (nx, ny); with S the conormal S n replaces n.
std::vector<Pair> boundary_pairs(int order, double nx, double ny, const double* g, const Aniso& S) {
  if (order == 4) {
    const double sx = S.on ? S.s11 * nx + S.s12 * ny : nx, sy = S.on ? S.s12 * nx + S.s22 * ny : ny;
    const Op I = op_I(), dn = op_dn(op_I(), sx, sy), lap = op_lapS(S), dnlap = op_dn(op_lapS(S), sx, sy);
    return {{I, I, g[0]}, {I, dnlap, 1.0}, {dnlap, I, 1.0}, {dn, dn, g[1]}, {dn, lap, -1.0}, {lap, dn, -1.0}};
  }
  const Op I = op_I(), dn = op_dn(op_I(), nx, ny), lap = op_lap(), dnlap = op_dn(op_lap(), nx, ny);
  const Op bil = op_bilap(), dnbil = op_dn(op_bilap(), nx, ny);
  return {{I, I, g[0]},   {I, dnbil, -1.0}, {dnbil, I, -1.0}, {dn, dn, g[1]},      {dn, bil, 1.0},
          {bil, dn, 1.0}, {lap, lap, g[2]}, {lap, dnlap, -1.0}, {dnlap, lap, -1.0}};
}

// (coefficient, x-order of v, y-order of v, x-order of u, y-order of u)
struct Term { double c; int vx, vy, ux, uy; };

std::vector<Term> expand(const std::vector<Pair>& ps) {
  std::vector<Term> t;
  for (auto& p : ps)
    for (auto& a : p.v)
      for (auto& b : p.u) t.push_back({p.c * a.c * b.c, a.ax, a.ay, b.ax, b.ay});
  return t;
}

}  // namespace

// ----------------------------------------------------------------------------- device

// packed term: coefficient, orders of v (x + 8 y) and of u (x + 8 y)
struct TermD { double c; int v, u; };

struct AsmArgs {
  int m, d, NP, NR;             // patches per side, block size, p+1, derivative orders stored
  const double* I;              // [(a*3 + da+1)][j][j'][r][r']
  const double* E0;             // [j][r] at x = 0 (patch 0)
  const double* E1;             // [j][r] at x = 1 (patch m-1)
  const int2* exps;             // basis k -> (x-degree, y-degree)
  const TermD* terms;           // interior terms, then the 4 edges
  int n_int, n_edge[4], off_edge[4];
};

__device__ __forceinline__ double Itab(const AsmArgs& A, int a, int da, int j, int jj, int r, int rr) {
  return A.I[((((int64_t)(a * 3 + da + 1) * A.NP + j) * A.NP + jj) * A.NR + r) * A.NR + rr];
}

__global__ void k_assemble_A(AsmArgs A, const int* __restrict__ row_of, const int* __restrict__ ci,
                             double* __restrict__ vals, int stride) {
  const int64_t blk = blockIdx.x;
  const int i = row_of[blk], j = ci[blk];
  const int m = A.m;
  const int ix = i % m, iy = i / m, jx = j % m, jy = j / m;
  const int dx = jx - ix, dy = jy - iy;
  const int dd = A.d * A.d;
  for (int e = threadIdx.x; e < dd; e += blockDim.x) {
    const int k = e / A.d, l = e - (e / A.d) * A.d;
    const int ka = A.exps[k].x, kb = A.exps[k].y, la = A.exps[l].x, lb = A.exps[l].y;
    double s = 0.0;
    for (int t = 0; t < A.n_int; ++t) {
      const TermD T = A.terms[t];
      const int v = T.v, u = T.u;
      s += T.c * Itab(A, ix, dx, ka, la, v & 7, u & 7) * Itab(A, iy, dy, kb, lb, v >> 3, u >> 3);
    }
    // edges x = 0, x = 1 (normal along x): point values in x, integral in y
    for (int side = 0; side < 2; ++side) {
      const int bp = side == 0 ? 0 : m - 1;
      if (ix != bp || jx != bp) continue;
      const double* E = side == 0 ? A.E0 : A.E1;
      for (int t = A.off_edge[side]; t < A.off_edge[side] + A.n_edge[side]; ++t) {
        const TermD T = A.terms[t];
        const int v = T.v, u = T.u;
        s += T.c * E[ka * A.NR + (v & 7)] * E[la * A.NR + (u & 7)] * Itab(A, iy, dy, kb, lb, v >> 3, u >> 3);
      }
    }
    // edges y = 0, y = 1
    for (int side = 0; side < 2; ++side) {
      const int bp = side == 0 ? 0 : m - 1;
      if (iy != bp || jy != bp) continue;
      const double* E = side == 0 ? A.E0 : A.E1;
      for (int t = A.off_edge[2 + side]; t < A.off_edge[2 + side] + A.n_edge[2 + side]; ++t) {
        const TermD T = A.terms[t];
        const int v = T.v, u = T.u;
        s += T.c * Itab(A, ix, dx, ka, la, v & 7, u & 7) * E[kb * A.NR + (v >> 3)] * E[lb * A.NR + (u >> 3)];
      }
    }
    vals[blk * stride + e] = s;
  }
}

// b_(i,k) = sum_ab cs_ab F[ix][ka][a] F[iy][kb][b]
__global__ void k_assemble_b(int m, int d, int NP, int K, const double* __restrict__ F, const double* __restrict__ cs,
                             const int2* __restrict__ exps, double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * m * d) return;
  const int i = (int)(t / d), k = (int)(t - (t / d) * d);
  const int ix = i % m, iy = i / m;
  const int ka = exps[k].x, kb = exps[k].y;
  const double* fx = F + ((int64_t)ix * NP + ka) * K;
  const double* fy = F + ((int64_t)iy * NP + kb) * K;
  double s = 0.0;
  for (int a = 0; a < K; ++a) {
    double r = 0.0;
    for (int c = 0; c < K; ++c) r += cs[a * K + c] * fy[c];
    s += fx[a] * r;
  }
  b[t] = s;
}

// P block (i, J) entry ((ka,kb),(la,lb)) = T[ix][slot_x][ka][la] * T[iy][slot_y][kb][lb]
__global__ void k_assemble_P(int m_f, int m_c, int d, int NP, const double* __restrict__ T,
                             const int* __restrict__ slot_of, const int* __restrict__ row_of,
                             const int* __restrict__ ci, const int2* __restrict__ exps, double* __restrict__ vals,
                             int stride) {
  const int64_t blk = blockIdx.x;
  const int i = row_of[blk], J = ci[blk];
  const int ix = i % m_f, iy = i / m_f, bx = J % m_c, by = J / m_c;
  const int sx = slot_of[ix * m_c + bx], sy = slot_of[iy * m_c + by];
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int k = e / d, l = e - (e / d) * d;
    const double tx = T[(((int64_t)ix * 2 + sx) * NP + exps[k].x) * NP + exps[l].x];
    const double ty = T[(((int64_t)iy * 2 + sy) * NP + exps[k].y) * NP + exps[l].y];
    vals[blk * stride + e] = tx * ty;
  }
}

// ----------------------------------------------------------------------------- host driver

namespace {

std::vector<int2> exponents(int p) {
  std::vector<int2> e;
  for (int s = 0; s <= p; ++s)
    for (int b = 0; b <= s; ++b) e.push_back(make_int2(s - b, b));
  return e;
}

template <typename T> T* upload(const std::vector<T>& v, cudaStream_t s) {
  T* d = nullptr;
  PUM_CUDA(cudaMalloc(&d, sizeof(T) * std::max<size_t>(v.size(), 1)));
  if (!v.empty()) PUM_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  return d;
}

std::vector<int> row_of_blocks(const std::vector<int>& rp) {
  std::vector<int> r(rp.back());
  for (size_t i = 0; i + 1 < rp.size(); ++i)
    for (int b = rp[i]; b < rp[i + 1]; ++b) r[b] = (int)i;
  return r;
}

}  // namespace

void assemble_finest(pum_ctx* ctx, const pum_problem& pr, Level& L, double* b_dev) {
  const int m = pr.finest_m, p = pr.p, order = pr.equation;
  const int d = (p + 1) * (p + 2) / 2, NP = p + 1, NR = order;  // derivative orders 0..order-1
  const int q = pr.quad_pts > 0 ? pr.quad_pts : p + 6;
  const double h = 1.0 / m;
  static const double defaults4[3] = {4.0, 2.0, 0.0}, defaults6[3] = {1.0e4, 1.0e2, 1.0};
  double gamma[3] = {0, 0, 0};
  for (int j = 0; j < order / 2; ++j) {
    const double C = pr.nitsche_c[j] > 0 ? pr.nitsche_c[j] : (order == 4 ? defaults4[j] : defaults6[j]);
    gamma[j] = C * (p + 1) * (p + 1) * std::pow(h, -(order - 1 - 2 * j));
  }
  Aniso S;
  S.on = !(pr.aniso[0] == 0.0 && pr.aniso[1] == 0.0 && pr.aniso[2] == 0.0) &&
         !(pr.aniso[0] == 1.0 && pr.aniso[1] == 0.0 && pr.aniso[2] == 1.0);
  if (S.on) {
    S.s11 = pr.aniso[0];
    S.s12 = pr.aniso[1];
    S.s22 = pr.aniso[2];
    PUM_CHECK(order == 4, PUM_ERR_INVALID_ARG, "anisotropy is defined for the biharmonic equation only");
    PUM_CHECK(S.s11 > 0.0 && S.s22 > 0.0 && S.s11 * S.s22 - S.s12 * S.s12 > 0.0, PUM_ERR_INVALID_ARG,
              "the anisotropy tensor must be SPD");
    // the consistency terms carry S twice against the u v penalty: gamma^(0) *= |S|_2^2
    const double half = 0.5 * (S.s11 + S.s22), rad = std::sqrt(0.25 * (S.s11 - S.s22) * (S.s11 - S.s22) + S.s12 * S.s12);
    gamma[0] *= (half + rad) * (half + rad);
  }
  Level1D L1(m);
  Basis1D B(p, NR);
  std::vector<double> gx, gw;
  gauss_legendre(q, gx, gw);
  const auto bp = L1.breakpoints();
  const int K = pr.f_coef ? pr.f_modes : 0;

  // 1-D tables
  std::vector<double> I((size_t)m * 3 * NP * NP * NR * NR, 0.0), F((size_t)m * NP * std::max(K, 1), 0.0);
  std::vector<double> X;  // per sub-interval values
  for (size_t s = 0; s + 1 < bp.size(); ++s) {
    const double lo = bp[s], hi = bp[s + 1];
    std::vector<int> act;
    for (int a = 0; a < m; ++a)
      if (L1.covers(a, lo, hi)) act.push_back(a);
    std::vector<double> x(q), w(q);
    for (int k = 0; k < q; ++k) {
      x[k] = 0.5 * (hi - lo) * gx[k] + 0.5 * (hi + lo);
      w[k] = 0.5 * (hi - lo) * gw[k];
    }
    // values[a_idx][j][r][k]
    std::vector<double> val(act.size() * NP * NR * q);
    for (size_t ai = 0; ai < act.size(); ++ai)
      for (int j = 0; j < NP; ++j)
        for (int r = 0; r < NR; ++r)
          for (int k = 0; k < q; ++k) val[((ai * NP + j) * NR + r) * q + k] = factor(L1, B, act[ai], j, x[k], r);
    for (size_t ai = 0; ai < act.size(); ++ai)
      for (size_t bi = 0; bi < act.size(); ++bi) {
        const int a = act[ai], da = act[bi] - act[ai];
        if (da < -1 || da > 1) continue;
        for (int j = 0; j < NP; ++j)
          for (int jj = 0; jj < NP; ++jj)
            for (int r = 0; r < NR; ++r)
              for (int rr = 0; rr < NR; ++rr) {
                double acc = 0.0;
                for (int k = 0; k < q; ++k)
                  acc += w[k] * val[((ai * NP + j) * NR + r) * q + k] * val[((bi * NP + jj) * NR + rr) * q + k];
                I[((((size_t)(a * 3 + da + 1) * NP + j) * NP + jj) * NR + r) * NR + rr] += acc;
              }
      }
    for (size_t ai = 0; ai < act.size(); ++ai)
      for (int j = 0; j < NP; ++j)
        for (int md = 1; md <= K; ++md) {
          double acc = 0.0;
          for (int k = 0; k < q; ++k) acc += w[k] * std::sin(md * M_PI * x[k]) * val[((ai * NP + j) * NR + 0) * q + k];
          F[((size_t)act[ai] * NP + j) * K + (md - 1)] += acc;
        }
  }
  std::vector<double> E0(NP * NR), E1(NP * NR);
  for (int j = 0; j < NP; ++j)
    for (int r = 0; r < NR; ++r) {
      E0[j * NR + r] = factor(L1, B, 0, j, 0.0, r);
      E1[j * NR + r] = factor(L1, B, m - 1, j, 1.0, r);
    }

  // term lists
  std::vector<TermD> terms;
  auto pack = [&](const std::vector<Term>& ts) {
    for (auto& t : ts) terms.push_back(TermD{t.c, t.vx + 8 * t.vy, t.ux + 8 * t.uy});
    return (int)ts.size();
  };
  AsmArgs A{};
  A.m = m; A.d = d; A.NP = NP; A.NR = NR;
  A.n_int = pack(expand(interior_pairs(order, S)));
  const double normals[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
  for (int e = 0; e < 4; ++e) {
    A.off_edge[e] = (int)terms.size();
    A.n_edge[e] = pack(expand(boundary_pairs(order, normals[e][0], normals[e][1], gamma, S)));
  }
  for (auto& t : terms) PUM_CHECK(t.v % 8 < NR && t.v / 8 < NR && t.u % 8 < NR && t.u / 8 < NR,
                                  PUM_ERR_INVALID_ARG, "assembly: derivative order beyond table");

  // 3 x 3 block stencil pattern (patches overlap iff |ix - jx| <= 1 and |iy - jy| <= 1)
  const int n = m * m;
  std::vector<int> rp(n + 1, 0), ci;
  for (int i = 0; i < n; ++i) {
    const int ix = i % m, iy = i / m;
    for (int jy = std::max(iy - 1, 0); jy <= std::min(iy + 1, m - 1); ++jy)
      for (int jx = std::max(ix - 1, 0); jx <= std::min(ix + 1, m - 1); ++jx) ci.push_back(jy * m + jx);
    rp[i + 1] = (int)ci.size();
  }
  L.m = m; L.n = n; L.d = d;
  bsr_alloc(L.A, n, n, d, PUM_F64, rp, ci);
  cudaStream_t s = ctx->stream;
  double* dI = upload(I, s);
  double* dE0 = upload(E0, s);
  double* dE1 = upload(E1, s);
  auto ex = exponents(p);
  int2* dex = upload(ex, s);
  TermD* dterms = upload(terms, s);
  int* drow = upload(row_of_blocks(rp), s);
  A.I = dI; A.E0 = dE0; A.E1 = dE1; A.exps = dex; A.terms = dterms;
  k_assemble_A<<<(unsigned)L.A.nnzb, 128, 0, s>>>(A, drow, L.A.col_idx, (double*)L.A.vals, L.A.stride);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  double *dF = nullptr, *dcs = nullptr;
  if (b_dev) {
    if (K > 0) {
      std::vector<double> cs(K * K);
      for (int a = 1; a <= K; ++a)
        for (int c = 1; c <= K; ++c)
          cs[(a - 1) * K + (c - 1)] = pr.f_coef[(a - 1) * K + (c - 1)] * std::pow((double)(a * a + c * c), -pr.f_decay / 2.0);
      dF = upload(F, s);
      dcs = upload(cs, s);
      const int64_t nt = (int64_t)n * d;
      k_assemble_b<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(m, d, NP, K, dF, dcs, dex, b_dev);
      count_launch(ctx);
      PUM_CUDA(cudaGetLastError());
    } else {
      PUM_CUDA(cudaMemsetAsync(b_dev, 0, sizeof(double) * (size_t)n * d, s));
    }
  }
  PUM_CUDA(cudaStreamSynchronize(s));
  for (void* ptr : {(void*)dI, (void*)dE0, (void*)dE1, (void*)dex, (void*)dterms, (void*)drow, (void*)dF, (void*)dcs})
    if (ptr) cudaFree(ptr);
}

// P of the fine level (m_f patches per side) from the coarse level m_f/2 by the
// global-to-local L2 projection of Section 4: with Legendre bases on the clipped boxes the
// local mass matrices are diagonal, and P_(i,J) = Tx (x) Ty with
// T[a][b][j][j'] = (2j+1)/w_a int_{box_a} P_j(xi_a) X^c_{b,j'} dx.
void build_prolongation(pum_ctx* ctx, int m_f, int p, int q, Level& fine) {
  PUM_CHECK(m_f % 2 == 0, PUM_ERR_INVALID_ARG, "prolongation: odd patch count");
  const int m_c = m_f / 2, NP = p + 1, d = (p + 1) * (p + 2) / 2;
  if (q <= 0) q = p + 6;
  Level1D Lf(m_f), Lc(m_c);
  Basis1D B(p, 0);
  std::vector<double> gx, gw;
  gauss_legendre(q, gx, gw);
  std::vector<double> cuts = Lf.breakpoints();
  for (double c : Lc.breakpoints()) cuts.push_back(c);
  std::sort(cuts.begin(), cuts.end());
  cuts.erase(std::unique(cuts.begin(), cuts.end()), cuts.end());

  std::vector<double> T((size_t)m_f * 2 * NP * NP, 0.0);
  std::vector<int> slot_of((size_t)m_f * m_c, -1);
  std::vector<std::vector<int>> coarse_of(m_f);
  for (int a = 0; a < m_f; ++a) {
    const double lo = Lf.lo(a), hi = Lf.hi(a), wa = hi - lo;
    for (int b = 0; b < m_c; ++b) {
      const double ov = std::min(hi, Lc.hi(b)) - std::max(lo, Lc.lo(b));
      if (ov > 0.0) coarse_of[a].push_back(b);
    }
    PUM_CHECK(coarse_of[a].size() <= 2, PUM_ERR_INVALID_ARG, "prolongation: more than 2 coarse patches");
    for (size_t sl = 0; sl < coarse_of[a].size(); ++sl) slot_of[(size_t)a * m_c + coarse_of[a][sl]] = (int)sl;
    std::vector<double> grid{lo};
    for (double c : cuts)
      if (c > lo && c < hi) grid.push_back(c);
    grid.push_back(hi);
    for (size_t u = 0; u + 1 < grid.size(); ++u)
      for (int k = 0; k < q; ++k) {
        const double x = 0.5 * (grid[u + 1] - grid[u]) * gx[k] + 0.5 * (grid[u + 1] + grid[u]);
        const double w = 0.5 * (grid[u + 1] - grid[u]) * gw[k];
        for (size_t sl = 0; sl < coarse_of[a].size(); ++sl) {
          const int b = coarse_of[a][sl];
          for (int j = 0; j < NP; ++j) {
            const double th = B.local(j, lo, hi, x, 0);
            for (int jj = 0; jj < NP; ++jj)
              T[(((size_t)a * 2 + sl) * NP + j) * NP + jj] += w * th * factor(Lc, B, b, jj, x, 0) * (2.0 * j + 1.0) / wa;
          }
        }
      }
  }
  const int n_f = m_f * m_f, n_c = m_c * m_c;
  std::vector<int> rp(n_f + 1, 0), ci;
  for (int i = 0; i < n_f; ++i) {
    const int ix = i % m_f, iy = i / m_f;
    for (int by : coarse_of[iy])
      for (int bx : coarse_of[ix]) ci.push_back(by * m_c + bx);
    rp[i + 1] = (int)ci.size();
  }
  bsr_alloc(fine.P, n_f, n_c, d, PUM_F64, rp, ci);
  cudaStream_t s = ctx->stream;
  double* dT = upload(T, s);
  int* dslot = upload(slot_of, s);
  int* drow = upload(row_of_blocks(rp), s);
  auto ex = exponents(p);
  int2* dex = upload(ex, s);
  k_assemble_P<<<(unsigned)fine.P.nnzb, 128, 0, s>>>(m_f, m_c, d, NP, dT, dslot, drow, fine.P.col_idx, dex,
                                                     (double*)fine.P.vals, fine.P.stride);
  count_launch(ctx);
  PUM_CUDA(cudaGetLastError());
  PUM_CUDA(cudaStreamSynchronize(s));
  for (void* ptr : {(void*)dT, (void*)dslot, (void*)drow, (void*)dex}) cudaFree(ptr);
}

}  // namespace pum
