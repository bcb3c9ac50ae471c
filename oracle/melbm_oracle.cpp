// melbm_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU restatement of the moment-encoded lattice Boltzmann
// (HOME-LBM) update of arXiv 2602.05295, written from the paper's equations so
// that the CUDA path can be checked against it.  Only tests, the smoke check and
// the benchmark's CPU-baseline leg may load this library; the product never does.
// It shares no code, header, table or constant with the CUDA path.
//
// Every routine follows the paper's definitions in the paper's order, with no
// blocking, fusion or reordering beyond what is stated next to it:
//   * lattice:        D3Q27, c_i in {-1,0,1}^3, w = product of 1D weights
//                     (2/3 at rest, 1/6 moving), c_s^2 = 1/3          (Sec. 3.1, App. D)
//   * collision:      moment-space HOME collision with forcing         (App. A)
//   * reconstruction: third-order Hermite expansion h(rho,u,S)         (Sec. 3.2, Eq. three_order_f)
//   * streaming:      pull form f_i(x) = f+_i(x - c_i)                 (Eq. streaming; Alg. 2)
//   * moments:        rho, rho u (+F/2), rho S                          (Eq. rho_u_stress)
//   * boundaries:     halfway bounce-back f_i(x) = f+_{opp(i)}(x) for solid
//                     links, equilibrium inflow, zero-gradient outflow  (split-kernel design, Sec. 4.2);
//                     or the moment-based reconstruction at moving solid walls,
//                     and the momentum-exchange force and torque  (Sec. 3.2, solid coupling)
//   * codec:          range, normalisation, dithered rounding to 16 bits (Sec. 5.4)
//   * D3Q19:          the same moments and collision on the 19-velocity lattice
//                     (Table 1's D3Q19 scene), periodic, with the third-order
//                     reconstruction projected on what that lattice carries
//
// Readings of the paper that it takes (each is also listed in the design notes):
//   * the xyz third-order Hermite term carries 1/c_s^6 (the other six triples
//     carry 1/(2 c_s^6)), which is the reading under which the reconstruction
//     reproduces its own third moments; `literal_xyz` selects the printed factor.
//   * the public state is the post-streaming (rho, u, S) at integer time (Alg. 2).
//   * S is the per-mass Hermite second moment, so its equilibrium is u u.
//   * the forcing terms of App. A are applied literally, with F at the colliding
//     and at the recovering cell.
//
// Parity pins: every function here is pinned by a CPU test against closed
// forms, invariants, symmetries or brute force (tests/test_oracle_pins.py).
// The amplification matrix G(k) that the oracle can build by complex step is
// pinned only through its closed-form limits; the paper's own analytic 2D
// matrices are not rebuilt ("parity unpinned" for those).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ----------------------------------------------------------------------------
// Lattice (Sec. 3.1).  Direction index i = (cx+1) + 3 (cy+1) + 9 (cz+1);
// the rest direction is i = 13 and the opposite of i is 26 - i.
// ----------------------------------------------------------------------------
constexpr double CS2 = 1.0 / 3.0;

struct Lattice {
  int c[27][3];
  double w[27];
  Lattice() {
    for (int i = 0; i < 27; ++i) {
      c[i][0] = i % 3 - 1;
      c[i][1] = (i / 3) % 3 - 1;
      c[i][2] = i / 9 - 1;
      double wi = 1.0;
      for (int a = 0; a < 3; ++a) wi *= (c[i][a] == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
      w[i] = wi;
    }
  }
};
const Lattice L;

inline int opposite(int i) { return 26 - i; }

// Symmetric 3x3 tensor stored as (xx, yy, zz, xy, xz, yz).
inline int sidx(int a, int b) {
  if (a == b) return a;
  if (a > b) { int t = a; a = b; b = t; }
  return (a == 0) ? (b == 1 ? 3 : 4) : 5;
}

template <class T>
struct Mom {  // rho, u_alpha, S_alphabeta (per-mass Hermite second moment)
  T rho;
  T u[3];
  T S[6];
};

// Cell types (priority SOLID > INFLOW > OUTFLOW > FLUID_BOUNDARY > FLUID).
enum : uint8_t { FLUID = 0, FLUID_BOUNDARY = 1, INFLOW = 2, OUTFLOW = 3, SOLID = 4 };

// ----------------------------------------------------------------------------
// Collision in moment space with forcing (App. A, Eqs. ourmomentcollision_*).
// Input: the post-streaming moments (rho*, u*, S*) of one cell and the force F.
// ----------------------------------------------------------------------------
template <class T>
Mom<T> collide(const Mom<T>& m, const T F[3], double tau) {
  Mom<T> o;
  const T rho = m.rho;
  o.rho = rho;                                                  // rho(t+1) = rho*
  for (int a = 0; a < 3; ++a) o.u[a] = m.u[a] + F[a] / (2.0 * rho);  // u + F/(2 rho)
  // Off-diagonal: (1 - 1/tau) S* + u*u*/tau + (2tau-1)/(2 tau rho) (F_a u_b + F_b u_a)
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      o.S[sidx(a, b)] = (1.0 - 1.0 / tau) * m.S[sidx(a, b)] + m.u[a] * m.u[b] / tau +
                        (2.0 * tau - 1.0) / (2.0 * tau * rho) * (F[a] * m.u[b] + F[b] * m.u[a]);
    }
  // Diagonal, with (b, g) the two other axes.
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, g = (a + 2) % 3;
    const T Saa = m.S[a], Sbb = m.S[b], Sgg = m.S[g];
    const T ua = m.u[a], ub = m.u[b], ug = m.u[g];
    o.S[a] = (tau - 1.0) / (3.0 * tau) * (2.0 * Saa - Sbb - Sgg) +
             (1.0 / 3.0) * (ua * ua + ub * ub + ug * ug) +
             (1.0 / (3.0 * tau)) * (2.0 * ua * ua - ub * ub - ug * ug) + F[a] * ua / rho +
             (tau - 1.0) / (3.0 * tau * rho) * (2.0 * F[a] * ua - F[b] * ub - F[g] * ug);
  }
  return o;
}

// ----------------------------------------------------------------------------
// Third-order Hermite reconstruction h_i(rho, u, S) (Eq. three_order_f).
//   f_i = rho w_i [1 + c.u/cs2 + H2(c):S/(2 cs2^2) + sum_{abg} k_abg H3_abg(c) T_abg]
//   T_abg = S_ab u_g + S_ag u_b + S_bg u_a - 2 u_a u_b u_g
// over the triples xxy, xyy, xxz, xzz, yzz, yyz, xyz.  k = 1/(2 cs2^3) for the
// six triples with a repeated index and 1/cs2^3 for xyz (see header), or the
// printed 1/(2 cs2^3) for all seven when literal_xyz is set.
// ----------------------------------------------------------------------------
inline double H2(int a, int b, const int* c) { return c[a] * c[b] - (a == b ? CS2 : 0.0); }
inline double H3(int a, int b, int g, const int* c) {
  return c[a] * c[b] * c[g] -
         CS2 * (c[a] * (b == g ? 1 : 0) + c[b] * (a == g ? 1 : 0) + c[g] * (a == b ? 1 : 0));
}
template <class T>
T Tabg(const Mom<T>& m, int a, int b, int g) {
  return m.S[sidx(a, b)] * m.u[g] + m.S[sidx(a, g)] * m.u[b] + m.S[sidx(b, g)] * m.u[a] -
         2.0 * m.u[a] * m.u[b] * m.u[g];
}
const int TRIPLES[7][3] = {{0, 0, 1}, {0, 1, 1}, {0, 0, 2}, {0, 2, 2}, {1, 2, 2}, {1, 1, 2}, {0, 1, 2}};

template <class T>
T reconstruct(int i, const Mom<T>& m, int literal_xyz) {
  const int* c = L.c[i];
  T cu = 0.0;
  for (int a = 0; a < 3; ++a) cu += double(c[a]) * m.u[a];
  T h2 = 0.0;  // H2:S summed over all nine (a, b)
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) h2 += H2(a, b, c) * m.S[sidx(a, b)];
  T h3 = 0.0;
  for (int t = 0; t < 7; ++t) {
    const int a = TRIPLES[t][0], b = TRIPLES[t][1], g = TRIPLES[t][2];
    const bool xyz = (t == 6);
    const double k = (xyz && !literal_xyz) ? 1.0 / (CS2 * CS2 * CS2) : 1.0 / (2.0 * CS2 * CS2 * CS2);
    h3 += k * H3(a, b, g, c) * Tabg(m, a, b, g);
  }
  return m.rho * L.w[i] * (1.0 + cu / CS2 + h2 / (2.0 * CS2 * CS2) + h3);
}

// ----------------------------------------------------------------------------
// Moments of the streamed populations (Eq. rho_u_stress):
//   rho = sum f, rho u = sum c f + F/2, rho S_ab = sum (c_a c_b - cs2 delta_ab) f.
// ----------------------------------------------------------------------------
template <class T>
Mom<T> moments(const T* f, const T F[3]) {
  Mom<T> o;
  T rho = 0.0, J[3] = {0.0, 0.0, 0.0}, P[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < 27; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) J[a] += double(L.c[i][a]) * f[i];
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) P[sidx(a, b)] += H2(a, b, L.c[i]) * f[i];
  }
  o.rho = rho;
  for (int a = 0; a < 3; ++a) o.u[a] = (J[a] + 0.5 * F[a]) / rho;
  for (int k = 0; k < 6; ++k) o.S[k] = P[k] / rho;
  return o;
}

// ----------------------------------------------------------------------------
// Grid helpers.  Linear index n = x + nx (y + ny z); SoA with 10 components
// (rho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz), component-major.
// ----------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;
  int64_t N() const { return int64_t(nx) * ny * nz; }
  int64_t idx(int x, int y, int z) const { return x + int64_t(nx) * (y + int64_t(ny) * z); }
  // x - c_i with periodic wrap
  int64_t pull_src(int64_t n, int i) const {
    int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (int64_t(nx) * ny));
    x = (x - L.c[i][0] + nx) % nx;
    y = (y - L.c[i][1] + ny) % ny;
    z = (z - L.c[i][2] + nz) % nz;
    return idx(x, y, z);
  }
};

template <class T>
Mom<T> load(const T* m, int64_t N, int64_t n) {
  Mom<T> o;
  o.rho = m[n];
  for (int a = 0; a < 3; ++a) o.u[a] = m[(1 + a) * N + n];
  for (int k = 0; k < 6; ++k) o.S[k] = m[(4 + k) * N + n];
  return o;
}
template <class T>
void store(T* m, int64_t N, int64_t n, const Mom<T>& v) {
  m[n] = v.rho;
  for (int a = 0; a < 3; ++a) m[(1 + a) * N + n] = v.u[a];
  for (int k = 0; k < 6; ++k) m[(4 + k) * N + n] = v.S[k];
}
template <class T>
void load_force(const T* F, int64_t N, int64_t n, T out[3]) {
  for (int a = 0; a < 3; ++a) out[a] = F ? F[a * N + n] : T(0.0);
}

// Solid walls (Sec. 3.2, solid coupling).  model 0: halfway bounce-back.
// model 1: the moment-based reconstruction: a link of fluid node x that meets a
// solid at p (the halfway point x - c_i / 2) receives the population
// h_i(rho^p, u^p, S^p) with rho^p = rho^x, u^p the velocity of the solid at p and
// S^p = u^p u^p + (S^x - u^x u^x), (rho, u, S)^x the post-collision moments of x.
// Solid cells belong to bodies (the mask value, 1..255); body b moves rigidly,
// u^p = V_b + Om_b x (p - r0_b), from table[9 b .. 9 b + 8] = (V, Om, r0).
struct WallSpec {
  int model;
  const uint8_t* body;   // N body ids (NULL: every solid is body 1)
  const double* table;   // 256 x 9
};

inline void wall_point(const Grid& g, int64_t n, int i, double p[3]) {
  const int x = int(n % g.nx), y = int((n / g.nx) % g.ny), z = int(n / (int64_t(g.nx) * g.ny));
  p[0] = x - 0.5 * L.c[i][0];
  p[1] = y - 0.5 * L.c[i][1];
  p[2] = z - 0.5 * L.c[i][2];
}

inline void wall_velocity(const WallSpec& w, int body, const double p[3], double up[3]) {
  const double* t = w.table + 9 * body;
  const double r[3] = {p[0] - t[6], p[1] - t[7], p[2] - t[8]};
  up[0] = t[0] + t[4] * r[2] - t[5] * r[1];
  up[1] = t[1] + t[5] * r[0] - t[3] * r[2];
  up[2] = t[2] + t[3] * r[1] - t[4] * r[0];
}

// (rho^p, u^p, S^p) of the moment-based reconstruction.
template <class T>
Mom<T> wall_moments(const Mom<T>& mx, const double up[3]) {
  Mom<T> o;
  o.rho = mx.rho;
  for (int a = 0; a < 3; ++a) o.u[a] = up[a];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b)
      o.S[sidx(a, b)] = up[a] * up[b] + (mx.S[sidx(a, b)] - mx.u[a] * mx.u[b]);
  return o;
}

// The population that solid link i of cell n receives.
template <class T>
T wall_population(const Grid& g, const std::vector<Mom<T>>& mp, int64_t n, int64_t src, int i,
                  const WallSpec* w, int literal_xyz) {
  if (!w || w->model == 0) return reconstruct(opposite(i), mp[n], literal_xyz);  // bounce-back
  double p[3], up[3];
  wall_point(g, n, i, p);
  wall_velocity(*w, w->body ? w->body[src] : 1, p, up);
  return reconstruct(i, wall_moments(mp[n], up), literal_xyz);
}

// The update of one non-solid cell from the post-collision moments `mp`
// (Alg. 2 streaming + moments, with the wall population for solid links).
template <class T>
Mom<T> pull_and_moments(const Grid& g, const std::vector<Mom<T>>& mp, const uint8_t* type,
                        const T* F, int64_t n, int literal_xyz, const WallSpec* w = nullptr) {
  T f[27];
  for (int i = 0; i < 27; ++i) {
    const int64_t src = g.pull_src(n, i);
    if (type && type[src] == SOLID)
      f[i] = wall_population(g, mp, n, src, i, w, literal_xyz);
    else
      f[i] = reconstruct(i, mp[src], literal_xyz);
  }
  T Fx[3];
  load_force(F, g.N(), n, Fx);
  return moments(f, Fx);
}

template <class T>
Mom<T> inflow_state(const double* inflow) {
  Mom<T> o;
  o.rho = inflow[0];
  for (int a = 0; a < 3; ++a) o.u[a] = inflow[1 + a];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) o.S[sidx(a, b)] = inflow[1 + a] * inflow[1 + b];
  return o;
}

// Deliberately wrong special-cell rules, selectable only through
// orc_step_planted_f64 so that the tests can show that their pins reject them:
//   PLANT_OUT_FROM_OLD   outflow copies the pre-step state of (nx-2, y, z);
//   PLANT_OUT_FROM_SELF  outflow copies x = nx-1 itself (no copy at all);
//   PLANT_IN_S_ZERO      inflow resets S to 0 instead of u_in u_in.
enum { PLANT_NONE = 0, PLANT_OUT_FROM_OLD = 1, PLANT_OUT_FROM_SELF = 2, PLANT_IN_S_ZERO = 3 };

// One full step over the grid.  Pass 1 collides every non-solid cell; pass 2
// pulls and re-forms the moments; pass 3 applies the zero-gradient outflow copy.
template <class T>
void step_grid(const Grid& g, double tau, const T* m, const T* F, const uint8_t* type,
               const double* inflow, T* out, int literal_xyz, const WallSpec* w = nullptr,
               int planted = PLANT_NONE) {
  const int64_t N = g.N();
  std::vector<Mom<T>> mp(N);
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    if (type && type[n] == SOLID) continue;
    T Fx[3];
    load_force(F, N, n, Fx);
    mp[n] = collide(load(m, N, n), Fx, tau);
  }
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    const uint8_t t = type ? type[n] : FLUID;
    if (t == SOLID) {
      store(out, N, n, load(m, N, n));  // solid cells keep their value
    } else if (t == INFLOW) {
      Mom<T> v = inflow_state<T>(inflow);
      if (planted == PLANT_IN_S_ZERO)
        for (int k = 0; k < 6; ++k) v.S[k] = T(0.0);
      store(out, N, n, v);
    } else {
      store(out, N, n, pull_and_moments(g, mp, type, F, n, literal_xyz, w));
    }
  }
  if (type && planted != PLANT_OUT_FROM_SELF) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
      if (type[n] != OUTFLOW) continue;
      const int64_t s = n - 1;  // (nx-2, y, z): the outflow plane is x = nx-1
      store(out, N, n, load(planted == PLANT_OUT_FROM_OLD ? m : out, N, s));
    }
  }
}

// ----------------------------------------------------------------------------
// D3Q19 (Sec. 6.3, Table 1 "Yeahright (D3Q19)"): the 19 velocities with
// |c|^2 <= 2, weights 1/3, 1/18, 1/36, c_s^2 = 1/3.  The collision (App. A) and
// the moments (Eq. rho_u_stress) are the same.  The paper does not give the
// reconstruction on this lattice; the reading taken is the orthogonal projection
// of Eq. three_order_f on the polynomials the lattice carries: H3_xyz vanishes on
// every D3Q19 velocity, and H3_aab and H3_bgg (the two triples with the same
// single index b) are not orthogonal there, while their sum and difference are,
// with lattice norms 2 c_s^6 and 6 c_s^6.  So
//   f_i = rho w_i [1 + c.u/cs2 + H2:S/(2 cs2^2)
//           + sum_b ((T_aab + T_bgg) (H3_aab + H3_bgg) / (2 cs2^3)
//                  + (T_aab - T_bgg) (H3_aab - H3_bgg) / (6 cs2^3))],
// which reproduces rho, rho u, rho S and the six rho T_aab exactly.
// Direction index: the D3Q27 index i with |c_i|^2 <= 2, in ascending order.
// ----------------------------------------------------------------------------
struct Lattice19 {
  int c[19][3];
  double w[19];
  int opp[19];
  Lattice19() {
    int k = 0;
    for (int i = 0; i < 27; ++i) {
      const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
      if (cx * cx + cy * cy + cz * cz > 2) continue;
      c[k][0] = cx;
      c[k][1] = cy;
      c[k][2] = cz;
      const int n2 = cx * cx + cy * cy + cz * cz;
      w[k] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
      ++k;
    }
    for (int a = 0; a < 19; ++a)
      for (int b = 0; b < 19; ++b)
        if (c[b][0] == -c[a][0] && c[b][1] == -c[a][1] && c[b][2] == -c[a][2]) opp[a] = b;
  }
};
const Lattice19 L19;

// The three pairs of triples sharing the single index b: (a a b, b g g).
const int PAIRS19[3][2][3] = {{{0, 0, 1}, {1, 2, 2}},   // b = y: xxy, yzz
                              {{0, 1, 1}, {0, 2, 2}},   // b = x: xyy, xzz
                              {{0, 0, 2}, {1, 1, 2}}};  // b = z: xxz, yyz

template <class T>
T reconstruct19(int i, const Mom<T>& m) {
  const int* c = L19.c[i];
  T cu = 0.0;
  for (int a = 0; a < 3; ++a) cu += double(c[a]) * m.u[a];
  T h2 = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) h2 += H2(a, b, c) * m.S[sidx(a, b)];
  T h3 = 0.0;
  for (int p = 0; p < 3; ++p) {
    const int* t1 = PAIRS19[p][0];
    const int* t2 = PAIRS19[p][1];
    const T T1 = Tabg(m, t1[0], t1[1], t1[2]), T2 = Tabg(m, t2[0], t2[1], t2[2]);
    const double H1 = H3(t1[0], t1[1], t1[2], c), Hb = H3(t2[0], t2[1], t2[2], c);
    h3 += (T1 + T2) * (H1 + Hb) / (2.0 * CS2 * CS2 * CS2) +
          (T1 - T2) * (H1 - Hb) / (6.0 * CS2 * CS2 * CS2);
  }
  return m.rho * L19.w[i] * (1.0 + cu / CS2 + h2 / (2.0 * CS2 * CS2) + h3);
}

template <class T>
Mom<T> moments19(const T* f, const T F[3]) {
  Mom<T> o;
  T rho = 0.0, J[3] = {0.0, 0.0, 0.0}, P[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < 19; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) J[a] += double(L19.c[i][a]) * f[i];
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) P[sidx(a, b)] += H2(a, b, L19.c[i]) * f[i];
  }
  o.rho = rho;
  for (int a = 0; a < 3; ++a) o.u[a] = (J[a] + 0.5 * F[a]) / rho;
  for (int k = 0; k < 6; ++k) o.S[k] = P[k] / rho;
  return o;
}

// The population solid link i of cell n receives on the D3Q19 lattice: halfway
// bounce-back, or the D3Q19 reconstruction of the wall state (rho^p, u^p, S^p) at
// the link's halfway point (the same solid coupling as on D3Q27).
double wall_population19(const Grid& g, const std::vector<Mom<double>>& mp, int64_t n,
                         int64_t src, int i, const WallSpec* w) {
  if (!w || w->model == 0) return reconstruct19(L19.opp[i], mp[n]);
  const int x = int(n % g.nx), y = int((n / g.nx) % g.ny), z = int(n / (int64_t(g.nx) * g.ny));
  const double p[3] = {x - 0.5 * L19.c[i][0], y - 0.5 * L19.c[i][1], z - 0.5 * L19.c[i][2]};
  double up[3];
  wall_velocity(*w, w->body ? w->body[src] : 1, p, up);
  return reconstruct19(i, wall_moments(mp[n], up));
}

// One D3Q19 step: collide every non-solid cell, pull the 19 populations (halfway
// bounce-back f_i(x) = f+_opp(i)(x) where x - c_i is solid, or the moving-wall
// population), re-form the moments; inflow cells take the inflow equilibrium,
// solid cells keep their value and the outflow plane copies x = nx-2 (the same
// split-design boundaries as D3Q27).
Mom<double> pull_and_moments19(const Grid& g, const std::vector<Mom<double>>& mp,
                               const uint8_t* type, const double* F, int64_t n,
                               const WallSpec* w = nullptr) {
  const int x = int(n % g.nx), y = int((n / g.nx) % g.ny), z = int(n / (int64_t(g.nx) * g.ny));
  double f[19];
  for (int i = 0; i < 19; ++i) {
    const int sx = (x - L19.c[i][0] + g.nx) % g.nx, sy = (y - L19.c[i][1] + g.ny) % g.ny,
              sz = (z - L19.c[i][2] + g.nz) % g.nz;
    const int64_t src = g.idx(sx, sy, sz);
    if (type && type[src] == SOLID)
      f[i] = wall_population19(g, mp, n, src, i, w);
    else
      f[i] = reconstruct19(i, mp[src]);
  }
  double Fx[3];
  load_force(F, g.N(), n, Fx);
  return moments19(f, Fx);
}

void step_grid19(const Grid& g, double tau, const double* m, const double* F, const uint8_t* type,
                 const double* inflow, double* out, const WallSpec* w = nullptr) {
  const int64_t N = g.N();
  std::vector<Mom<double>> mp(N);
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    if (type && type[n] == SOLID) continue;
    double Fx[3];
    load_force(F, N, n, Fx);
    mp[n] = collide(load(m, N, n), Fx, tau);
  }
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    const uint8_t t = type ? type[n] : FLUID;
    if (t == SOLID)
      store(out, N, n, load(m, N, n));
    else if (t == INFLOW)
      store(out, N, n, inflow_state<double>(inflow));
    else
      store(out, N, n, pull_and_moments19(g, mp, type, F, n, w));
  }
  if (type) {
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n)
      if (type[n] == OUTFLOW) store(out, N, n, load(out, N, n - 1));
  }
}

// ----------------------------------------------------------------------------
// Hand-written reverse mode (vector-Jacobian products) of collide, reconstruct
// and moments, used by the discrete adjoint of one step.
// ----------------------------------------------------------------------------
// d(moments)/d(f, F) transposed: given (rho_bar, u_bar, S_bar) of the output.
inline void moments_vjp(const double* f, const double F[3], const Mom<double>& ob, double* fb,
                        double Fb[3]) {
  double rho = 0.0, J[3] = {0, 0, 0}, P[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 27; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) J[a] += L.c[i][a] * f[i];
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) P[sidx(a, b)] += H2(a, b, L.c[i]) * f[i];
  }
  for (int a = 0; a < 3; ++a) J[a] += 0.5 * F[a];
  // u = J/rho, S = P/rho
  double Jb[3], Pb[6], rhob = ob.rho;
  for (int a = 0; a < 3; ++a) {
    Jb[a] = ob.u[a] / rho;
    rhob -= ob.u[a] * J[a] / (rho * rho);
  }
  for (int k = 0; k < 6; ++k) {
    Pb[k] = ob.S[k] / rho;
    rhob -= ob.S[k] * P[k] / (rho * rho);
  }
  for (int i = 0; i < 27; ++i) {
    double s = rhob;
    for (int a = 0; a < 3; ++a) s += L.c[i][a] * Jb[a];
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) s += H2(a, b, L.c[i]) * Pb[sidx(a, b)];
    fb[i] = s;
  }
  for (int a = 0; a < 3; ++a) Fb[a] += 0.5 * Jb[a];
}

// d(h_i)/d(rho, u, S) transposed, accumulated into mb.
inline void reconstruct_vjp(int i, const Mom<double>& m, double fb, Mom<double>& mb, int literal_xyz) {
  const int* c = L.c[i];
  const double w = L.w[i];
  double cu = 0.0, h2 = 0.0, h3 = 0.0;
  for (int a = 0; a < 3; ++a) cu += c[a] * m.u[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) h2 += H2(a, b, c) * m.S[sidx(a, b)];
  double kt[7];
  for (int t = 0; t < 7; ++t) {
    const int a = TRIPLES[t][0], b = TRIPLES[t][1], g = TRIPLES[t][2];
    const double k = (t == 6 && !literal_xyz) ? 1.0 / (CS2 * CS2 * CS2) : 1.0 / (2.0 * CS2 * CS2 * CS2);
    kt[t] = k * H3(a, b, g, c);
    h3 += kt[t] * Tabg(m, a, b, g);
  }
  const double bracket = 1.0 + cu / CS2 + h2 / (2.0 * CS2 * CS2) + h3;
  // f = rho w bracket
  mb.rho += fb * w * bracket;
  const double gb = fb * m.rho * w;  // d f / d bracket
  for (int a = 0; a < 3; ++a) mb.u[a] += gb * c[a] / CS2;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) mb.S[sidx(a, b)] += gb * H2(a, b, c) / (2.0 * CS2 * CS2);
  for (int t = 0; t < 7; ++t) {
    const int a = TRIPLES[t][0], b = TRIPLES[t][1], g = TRIPLES[t][2];
    const double tb = gb * kt[t];  // d f / d T_abg
    // T = S_ab u_g + S_ag u_b + S_bg u_a - 2 u_a u_b u_g
    mb.S[sidx(a, b)] += tb * m.u[g];
    mb.S[sidx(a, g)] += tb * m.u[b];
    mb.S[sidx(b, g)] += tb * m.u[a];
    mb.u[g] += tb * (m.S[sidx(a, b)] - 2.0 * m.u[a] * m.u[b]);
    mb.u[b] += tb * (m.S[sidx(a, g)] - 2.0 * m.u[a] * m.u[g]);
    mb.u[a] += tb * (m.S[sidx(b, g)] - 2.0 * m.u[b] * m.u[g]);
  }
}

// d(collide)/d(m, F) transposed.
inline void collide_vjp(const Mom<double>& m, const double F[3], double tau, const Mom<double>& ob,
                        Mom<double>& mb, double Fb[3]) {
  const double rho = m.rho;
  mb.rho += ob.rho;
  for (int a = 0; a < 3; ++a) {  // u+ = u + F/(2 rho)
    mb.u[a] += ob.u[a];
    Fb[a] += ob.u[a] / (2.0 * rho);
    mb.rho += -ob.u[a] * F[a] / (2.0 * rho * rho);
  }
  for (int a = 0; a < 3; ++a)
    for (int b = a + 1; b < 3; ++b) {
      const double sb = ob.S[sidx(a, b)];
      const double kf = (2.0 * tau - 1.0) / (2.0 * tau);
      const double G = F[a] * m.u[b] + F[b] * m.u[a];
      mb.S[sidx(a, b)] += sb * (1.0 - 1.0 / tau);
      mb.u[a] += sb * (m.u[b] / tau + kf / rho * F[b]);
      mb.u[b] += sb * (m.u[a] / tau + kf / rho * F[a]);
      Fb[a] += sb * kf / rho * m.u[b];
      Fb[b] += sb * kf / rho * m.u[a];
      mb.rho += -sb * kf * G / (rho * rho);
    }
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, g = (a + 2) % 3;
    const double sb = ob.S[a];
    const double k1 = (tau - 1.0) / (3.0 * tau);
    mb.S[a] += sb * 2.0 * k1;
    mb.S[b] += -sb * k1;
    mb.S[g] += -sb * k1;
    const double ua = m.u[a], ub = m.u[b], ug = m.u[g];
    // (1/3)|u|^2 + (1/(3 tau))(2ua^2 - ub^2 - ug^2)
    mb.u[a] += sb * ((2.0 / 3.0) * ua + (4.0 / (3.0 * tau)) * ua);
    mb.u[b] += sb * ((2.0 / 3.0) * ub - (2.0 / (3.0 * tau)) * ub);
    mb.u[g] += sb * ((2.0 / 3.0) * ug - (2.0 / (3.0 * tau)) * ug);
    // F_a u_a / rho
    Fb[a] += sb * ua / rho;
    mb.u[a] += sb * F[a] / rho;
    mb.rho += -sb * F[a] * ua / (rho * rho);
    // (tau-1)/(3 tau rho) (2 F_a u_a - F_b u_b - F_g u_g)
    const double k2 = (tau - 1.0) / (3.0 * tau);
    const double Q = 2.0 * F[a] * ua - F[b] * ub - F[g] * ug;
    Fb[a] += sb * k2 / rho * 2.0 * ua;
    Fb[b] += -sb * k2 / rho * ub;
    Fb[g] += -sb * k2 / rho * ug;
    mb.u[a] += sb * k2 / rho * 2.0 * F[a];
    mb.u[b] += -sb * k2 / rho * F[b];
    mb.u[g] += -sb * k2 / rho * F[g];
    mb.rho += -sb * k2 * Q / (rho * rho);
  }
}

Mom<double> zero_mom() {
  Mom<double> z;
  z.rho = 0.0;
  for (int a = 0; a < 3; ++a) z.u[a] = 0.0;
  for (int k = 0; k < 6; ++k) z.S[k] = 0.0;
  return z;
}

// ----------------------------------------------------------------------------
// Counter-based dither generator: pcg4d of Jarzynski & Olano, "Hash Functions
// for GPU Rendering", JCGT 9(3), 2020, on the counter (x, y, z, t ^ seed).
// ----------------------------------------------------------------------------
inline void pcg4d(uint32_t v[4]) {
  for (int k = 0; k < 4; ++k) v[k] = v[k] * 1664525u + 1013904223u;
  v[0] += v[1] * v[3];
  v[1] += v[2] * v[0];
  v[2] += v[0] * v[1];
  v[3] += v[1] * v[2];
  for (int k = 0; k < 4; ++k) v[k] ^= v[k] >> 16;
  v[0] += v[1] * v[3];
  v[1] += v[2] * v[0];
  v[2] += v[0] * v[1];
  v[3] += v[1] * v[2];
}

// Ten dither values d_k in (0, 1) for one cell and one time index (reading 7 of
// the design notes: Sec. 5.4 fixes the noise -- zero-mean, uniform over one
// quantisation unit -- but not its source).  Every component takes a 16-bit field
// f: components 0..7 the low (even k) and high (odd k) halves of word k/2 of the
// hash, component 8 the low half of v0 xor v2 and component 9 the high half of
// v1 xor v3 (each uniform over the 2^16 fields, and independent of any single
// other component's field).  d = (f + 1/2) / 2^16: the midpoints of 2^16 equal
// cells of [0, 1), whose mean is exactly 1/2, so the added noise d - 1/2 is
// zero-mean as Sec. 5.4 requires.
inline int dither_bits(int) { return 16; }
inline float dither_of_field(int k, uint32_t field) {
  return (float(field) + 0.5f) / float(1u << dither_bits(k));
}
inline void dither_fields(uint32_t x, uint32_t y, uint32_t z, uint32_t t, uint32_t seed,
                          uint32_t f[10]) {
  uint32_t v[4] = {x, y, z, t ^ seed};
  pcg4d(v);
  for (int k = 0; k < 8; ++k) {
    const uint32_t w = v[k / 2];
    f[k] = (k % 2 == 0) ? (w & 0xFFFFu) : (w >> 16);
  }
  f[8] = (v[0] ^ v[2]) & 0xFFFFu;
  f[9] = (v[1] ^ v[3]) >> 16;
}
inline void dither10(uint32_t x, uint32_t y, uint32_t z, uint32_t t, uint32_t seed, float d[10]) {
  uint32_t f[10];
  dither_fields(x, y, z, t, seed, f);
  for (int k = 0; k < 10; ++k) d[k] = dither_of_field(k, f[k]);
}

// Stored-variable ranges (Sec. 5.4 moment range analysis and range reduction):
// rho in [0.8, 1.5]; u_a in [-0.4, 0.4]; rho S^neq_ab = rho (S_ab - u_a u_b) in [-0.1, 0.1].
const double QLO[10] = {0.8, -0.4, -0.4, -0.4, -0.1, -0.1, -0.1, -0.1, -0.1, -0.1};
const double QHI[10] = {1.5, 0.4, 0.4, 0.4, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1};

// The fixed-point map of Sec. 5.4, q = floor((m - m_min)/step + d) with
// step = (m_max - m_min)/(2^b - 1) and the dither d in [0, 1), taken in FP32 (the
// precision the kernels take this decision in).  It is evaluated relative to the
// code qc nearest to the centre of the values (rho = 1, u = 0, rho S^neq = 0),
// whose value is c = m_min + qc step:
//   w = m' K + b       with m' = rho - 1 for the density and m' = m otherwise,
//                      K = 1/step, b = (centre - m_min)/step - qc
//   q = qc + floor(clamp(w, -qc, 2^b - 1 - qc) + d)
//   decoded value  m' = c + (q - qc) step.
// This is the same formula in exact arithmetic; in FP32 the rounding of the
// constants then only scales the (zero-mean) deviation from the centre, and the
// floor of w + d is exact, so the rounding stays unbiased (Sec. 5.4 dithering).
// All constants are the FP32 roundings of their FP64 values.
// Bit widths of the adaptive allocation (Sec. 6.2.2, "b_rho_u / b_S"): rho and u
// (components 0..3) take b_ru bits, rho S^neq (components 4..9) b_s bits; the
// grid of component k has Q = 2^b - 1 steps.  16/16 is the default.
struct Bits {
  int ru = 16, s = 16;
};
inline double levels(int k, Bits bits) { return double((1u << (k < 4 ? bits.ru : bits.s)) - 1u); }

struct QGroup {
  double lo, hi, centre;  // range and centre in the shifted variable m'
  double qc, Q;           // centre code and number of steps
};
inline QGroup qgroup(int k, Bits bits) {
  QGroup g;
  const double shift = (k == 0) ? 1.0 : 0.0;
  g.lo = QLO[k] - shift;
  g.hi = QHI[k] - shift;
  g.centre = 0.0;
  g.Q = levels(k, bits);
  g.qc = std::floor((g.centre - g.lo) * g.Q / (g.hi - g.lo) + 0.5);
  return g;
}
inline float q_step(int k, Bits bits) {
  QGroup g = qgroup(k, bits);
  return float((g.hi - g.lo) / g.Q);
}
inline float q_K(int k, Bits bits) {
  QGroup g = qgroup(k, bits);
  return float(g.Q / (g.hi - g.lo));
}
inline float q_b(int k, Bits bits) {
  QGroup g = qgroup(k, bits);
  return float((g.centre - g.lo) * g.Q / (g.hi - g.lo) - g.qc);
}
inline float q_c(int k, Bits bits) {
  QGroup g = qgroup(k, bits);
  return float(g.lo + g.qc * (g.hi - g.lo) / g.Q);
}

// Encode the shifted value mp (rho - 1 for k = 0) with dither d.
inline uint16_t encode_one(float mp, int k, float d, Bits bits) {
  const QGroup g = qgroup(k, bits);
  float w = std::fma(mp, q_K(k, bits), q_b(k, bits));
  const float wlo = float(-g.qc), whi = float(g.Q - g.qc);
  w = std::fmax(w, wlo);  // fmax/fmin return the other operand for NaN: NaN -> code 0
  w = std::fmin(w, whi);
  const double f = std::floor(double(w) + double(d));  // exact in double
  return uint16_t(int(g.qc) + int(f));
}

// Dequantisation: m = c + (q - qc) step, returned for the unshifted variable
// (rho for k = 0), in FP64 from the FP32 grid constants.
inline double decode_one(uint16_t q, int k, Bits bits) {
  const QGroup g = qgroup(k, bits);
  const double shift = (k == 0) ? 1.0 : 0.0;
  return shift + double(q_c(k, bits)) + (double(q) - g.qc) * double(q_step(k, bits));
}

}  // namespace

// ============================================================================
// C interface for the Python test harness.
// ============================================================================
extern "C" {

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void orc_lattice(int* c /*27x3*/, double* w /*27*/) {
  for (int i = 0; i < 27; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
  }
}

// Per-cell primitives on arrays of cells (10 moments per cell, cell-major).
void orc_collide(int64_t ncell, const double* m, const double* F, double tau, double* out) {
  for (int64_t n = 0; n < ncell; ++n) {
    Mom<double> v = load(m + 10 * n, 1, 0);
    double Fx[3] = {F ? F[3 * n] : 0.0, F ? F[3 * n + 1] : 0.0, F ? F[3 * n + 2] : 0.0};
    store(out + 10 * n, 1, 0, collide(v, Fx, tau));
  }
}

void orc_reconstruct(int64_t ncell, const double* m, int literal_xyz, double* f /*27 per cell*/) {
  for (int64_t n = 0; n < ncell; ++n) {
    Mom<double> v = load(m + 10 * n, 1, 0);
    for (int i = 0; i < 27; ++i) f[27 * n + i] = reconstruct(i, v, literal_xyz);
  }
}

void orc_moments(int64_t ncell, const double* f, const double* F, double* out) {
  for (int64_t n = 0; n < ncell; ++n) {
    double Fx[3] = {F ? F[3 * n] : 0.0, F ? F[3 * n + 1] : 0.0, F ? F[3 * n + 2] : 0.0};
    store(out + 10 * n, 1, 0, moments(f + 27 * n, Fx));
  }
}

// Cell classification and boundary list (analogue of the surface marking of Sec. 4.2).
//   type: SOLID if mask; else INFLOW if inflow and x == 0; else OUTFLOW if outflow,
//   x == nx-1 and (nx-2, y, z) is not solid; else FLUID_BOUNDARY if any x - c_i is
//   solid (periodic wrap); else FLUID.
//   link: bit i set iff x - c_i is solid (0 for solid cells).
//   list: ascending linear index of INFLOW and FLUID_BOUNDARY cells; returns its length.
int64_t orc_classify(int nx, int ny, int nz, const uint8_t* mask, int inflow, int outflow,
                     uint8_t* type, uint32_t* link, uint32_t* list_cell, uint32_t* list_word) {
  Grid g{nx, ny, nz};
  const int64_t N = g.N();
  for (int64_t n = 0; n < N; ++n) {
    const int x = int(n % nx);
    uint32_t bits = 0;
    if (!mask[n]) {
      for (int i = 0; i < 27; ++i)
        if (mask[g.pull_src(n, i)]) bits |= (1u << i);
    }
    uint8_t t;
    if (mask[n]) t = SOLID;
    else if (inflow && x == 0) t = INFLOW;
    else if (outflow && x == nx - 1 && nx >= 2 && !mask[n - 1]) t = OUTFLOW;
    else if (bits) t = FLUID_BOUNDARY;
    else t = FLUID;
    type[n] = t;
    link[n] = bits;
  }
  int64_t L_ = 0;
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] == INFLOW || type[n] == FLUID_BOUNDARY) {
      if (list_cell) list_cell[L_] = uint32_t(n);
      if (list_word) list_word[L_] = (uint32_t(type[n]) << 27) | link[n];
      ++L_;
    }
  }
  return L_;
}

// One step on the whole grid, public state (rho, u, S) in FP64.
void orc_step_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                  const uint8_t* type, const double* inflow, int literal_xyz, double* out) {
  step_grid<double>(Grid{nx, ny, nz}, tau, m, F, type, inflow, out, literal_xyz);
}

// The same step with one of the PLANT_* mistakes of the special-cell rules (test
// ablation only; planted = 0 is orc_step_f64).
void orc_step_planted_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                          const uint8_t* type, const double* inflow, int planted, double* out) {
  step_grid<double>(Grid{nx, ny, nz}, tau, m, F, type, inflow, out, 0, nullptr, planted);
}

// One D3Q19 step (public state, component-major 10 x N; type and inflow as for
// the D3Q27 step, or NULL for a periodic box).
void orc_step19_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                    const uint8_t* type, const double* inflow, double* out) {
  step_grid19(Grid{nx, ny, nz}, tau, m, F, type, inflow, out);
}

// The D3Q19 update of the listed cells only (each collides the cells it pulls
// from; type / inflow as for the full step, or NULL); out is [ncells][10].
void orc_step19_cells_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                          const uint8_t* type, const double* inflow, const int64_t* cells,
                          int64_t ncells, double* out) {
  Grid g{nx, ny, nz};
  const int64_t N = g.N();
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < ncells; ++k) {
    int64_t n = cells[k];
    uint8_t t = type ? type[n] : FLUID;
    if (t == OUTFLOW) {
      n = n - 1;
      t = type[n];
    }
    Mom<double> r;
    if (t == SOLID) {
      r = load(m, N, n);
    } else if (t == INFLOW) {
      r = inflow_state<double>(inflow);
    } else {
      const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (int64_t(nx) * ny));
      double Fn[3];
      load_force(F, N, n, Fn);
      double f[19];
      for (int i = 0; i < 19; ++i) {
        const int sx = (x - L19.c[i][0] + nx) % nx, sy = (y - L19.c[i][1] + ny) % ny,
                  sz = (z - L19.c[i][2] + nz) % nz;
        const int64_t src = g.idx(sx, sy, sz);
        if (type && type[src] == SOLID) {
          f[i] = reconstruct19(L19.opp[i], collide(load(m, N, n), Fn, tau));
        } else {
          double Fx[3];
          load_force(F, N, src, Fx);
          f[i] = reconstruct19(i, collide(load(m, N, src), Fx, tau));
        }
      }
      r = moments19(f, Fn);
    }
    store(out + 10 * k, 1, 0, r);
  }
}

// The D3Q19 step with the wall model of WallSpec.
void orc_step19_wall_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                         const uint8_t* type, const double* inflow, int model,
                         const uint8_t* body, const double* table, double* out) {
  const WallSpec w{model, body, table};
  step_grid19(Grid{nx, ny, nz}, tau, m, F, type, inflow, out, &w);
}

// Force and torque on body `body_id` (0: every solid) by momentum exchange over
// the 19-velocity links, as orc_solid_force_f64 does over 27.
void orc_solid_force19_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                           const uint8_t* type, int model, const uint8_t* body,
                           const double* table, int body_id, double* out /*6*/) {
  const Grid g{nx, ny, nz};
  const int64_t N = g.N();
  const WallSpec w{model, body, table};
  std::vector<Mom<double>> mp(N);
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] == SOLID) continue;
    double Fx[3];
    load_force(F, N, n, Fx);
    mp[n] = collide(load(m, N, n), Fx, tau);
  }
  for (int k = 0; k < 6; ++k) out[k] = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] != FLUID_BOUNDARY) continue;
    const int x = int(n % nx), y = int((n / nx) % ny), z = int(n / (int64_t(nx) * ny));
    for (int i = 0; i < 19; ++i) {
      const int64_t src = g.idx((x - L19.c[i][0] + nx) % nx, (y - L19.c[i][1] + ny) % ny,
                                (z - L19.c[i][2] + nz) % nz);
      if (type[src] != SOLID) continue;
      const int b = body ? body[src] : 1;
      if (body_id && b != body_id) continue;
      const double f_out = reconstruct19(L19.opp[i], mp[n]);
      const double f_in = wall_population19(g, mp, n, src, i, &w);
      const double p[3] = {x - 0.5 * L19.c[i][0], y - 0.5 * L19.c[i][1], z - 0.5 * L19.c[i][2]};
      double dF[3];
      for (int a = 0; a < 3; ++a) dF[a] = -double(L19.c[i][a]) * (f_in + f_out);
      const double* t = table + 9 * (body_id ? body_id : b);
      const double r[3] = {p[0] - t[6], p[1] - t[7], p[2] - t[8]};
      out[0] += dF[0];
      out[1] += dF[1];
      out[2] += dF[2];
      out[3] += r[1] * dF[2] - r[2] * dF[1];
      out[4] += r[2] * dF[0] - r[0] * dF[2];
      out[5] += r[0] * dF[1] - r[1] * dF[0];
    }
  }
}

// D3Q19 populations of one moment set (rho, u[3], S[6]) and its 19 velocities
// and weights (for the moment-identity pins).
void orc_reconstruct19(const double* m10, double* f19, int* c57, double* w19) {
  Mom<double> m;
  m.rho = m10[0];
  for (int a = 0; a < 3; ++a) m.u[a] = m10[1 + a];
  for (int k = 0; k < 6; ++k) m.S[k] = m10[4 + k];
  for (int i = 0; i < 19; ++i) {
    f19[i] = reconstruct19(i, m);
    for (int a = 0; a < 3; ++a) c57[3 * i + a] = L19.c[i][a];
    w19[i] = L19.w[i];
  }
}

// The step with the wall model of WallSpec (body ids and the 256 x 9 motion table).
void orc_step_wall_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                       const uint8_t* type, const double* inflow, int model, const uint8_t* body,
                       const double* table, double* out) {
  const WallSpec w{model, body, table};
  step_grid<double>(Grid{nx, ny, nz}, tau, m, F, type, inflow, out, 0, &w);
}

// Force and torque (about r0 of the body) that the next step transfers to the
// solid cells of body `body_id` (0: every solid): momentum exchange over every
// solid link i of every FLUID_BOUNDARY cell x, -c_i (f_in + f_out), with f_out =
// h_opp(i)(x) the post-collision population leaving x towards the wall and f_in
// the population the wall returns; torque sum (p - r0) x that, p the link's
// halfway point.  FP64, fixed order.
void orc_solid_force_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                         const uint8_t* type, int model, const uint8_t* body, const double* table,
                         int body_id, double* out /*6*/) {
  const Grid g{nx, ny, nz};
  const int64_t N = g.N();
  const WallSpec w{model, body, table};
  std::vector<Mom<double>> mp(N);
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] == SOLID) continue;
    double Fx[3];
    load_force(F, N, n, Fx);
    mp[n] = collide(load(m, N, n), Fx, tau);
  }
  for (int k = 0; k < 6; ++k) out[k] = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    if (type[n] != FLUID_BOUNDARY) continue;
    for (int i = 0; i < 27; ++i) {
      const int64_t src = g.pull_src(n, i);
      if (type[src] != SOLID) continue;
      const int b = body ? body[src] : 1;
      if (body_id && b != body_id) continue;
      const double f_out = reconstruct(opposite(i), mp[n], 0);
      const double f_in = wall_population(g, mp, n, src, i, &w, 0);
      double dF[3], p[3];
      for (int a = 0; a < 3; ++a) dF[a] = -double(L.c[i][a]) * (f_in + f_out);
      wall_point(g, n, i, p);
      const double* t = table + 9 * (body_id ? body_id : b);
      const double r[3] = {p[0] - t[6], p[1] - t[7], p[2] - t[8]};
      out[0] += dF[0];
      out[1] += dF[1];
      out[2] += dF[2];
      out[3] += r[1] * dF[2] - r[2] * dF[1];
      out[4] += r[2] * dF[0] - r[0] * dF[2];
      out[5] += r[0] * dF[1] - r[1] * dF[0];
    }
  }
}

// The same step on complex numbers (interleaved re/im), for complex-step derivatives.
void orc_step_c128(int nx, int ny, int nz, double tau, const double* m, const double* F,
                   const uint8_t* type, const double* inflow, int literal_xyz, double* out) {
  using C = std::complex<double>;
  step_grid<C>(Grid{nx, ny, nz}, tau, reinterpret_cast<const C*>(m), reinterpret_cast<const C*>(F),
               type, inflow, reinterpret_cast<C*>(out), literal_xyz);
}

// The step evaluated at selected cells only (cell-major output, 10 per cell), for
// sampled checks on grids too large to step whole.  Outflow cells return the new
// value of (nx-2, y, z); solid cells their old value.
void orc_step_cells_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                        const uint8_t* type, const double* inflow, const int64_t* cells,
                        int64_t ncells, double* out) {
  Grid g{nx, ny, nz};
  const int64_t N = g.N();
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < ncells; ++k) {
    int64_t n = cells[k];
    uint8_t t = type ? type[n] : FLUID;
    if (t == OUTFLOW) {
      n = n - 1;
      t = type[n];
    }
    Mom<double> r;
    if (t == SOLID) {
      r = load(m, N, n);
    } else if (t == INFLOW) {
      r = inflow_state<double>(inflow);
    } else {
      // collide only the 27 cells this one pulls from
      double f[27];
      for (int i = 0; i < 27; ++i) {
        const int64_t src = g.pull_src(n, i);
        if (type && type[src] == SOLID) {
          double Fx[3];
          load_force(F, N, n, Fx);
          f[i] = reconstruct(opposite(i), collide(load(m, N, n), Fx, tau), 0);
        } else {
          double Fx[3];
          load_force(F, N, src, Fx);
          f[i] = reconstruct(i, collide(load(m, N, src), Fx, tau), 0);
        }
      }
      double Fx[3];
      load_force(F, N, n, Fx);
      r = moments(f, Fx);
    }
    store(out + 10 * k, 1, 0, r);
  }
}

// Discrete adjoint of one orc_step_f64 (vector-Jacobian product): given
// lam_out = dL/d(out), returns lam_in = dL/d(m) and adds dL/dF into gF (if gF).
void orc_step_vjp_f64(int nx, int ny, int nz, double tau, const double* m, const double* F,
                      const uint8_t* type, const double* lam_out, double* lam_in, double* gF) {
  Grid g{nx, ny, nz};
  const int64_t N = g.N();
  // Outflow copy (pass 3) reversed: the outflow cell's output came from (nx-2).
  std::vector<double> lo(lam_out, lam_out + 10 * N);
  if (type) {
    for (int64_t n = 0; n < N; ++n) {
      if (type[n] != OUTFLOW) continue;
      for (int k = 0; k < 10; ++k) {
        lo[k * N + n - 1] += lo[k * N + n];
        lo[k * N + n] = 0.0;
      }
    }
  }
  // Forward quantities: post-collision moments.
  std::vector<Mom<double>> mp(N);
  for (int64_t n = 0; n < N; ++n) {
    if (type && type[n] == SOLID) continue;
    double Fx[3];
    load_force(F, N, n, Fx);
    mp[n] = collide(load(m, N, n), Fx, tau);
  }
  // Pass 2 reversed: scatter population adjoints onto the post-collision moments.
  std::vector<Mom<double>> mpb(N, zero_mom());
  std::vector<double> Fb(3 * N, 0.0);
  for (int64_t n = 0; n < N; ++n) {
    const uint8_t t = type ? type[n] : FLUID;
    if (t == SOLID) {
      for (int k = 0; k < 10; ++k) lam_in[k * N + n] = lo[k * N + n];  // identity
      continue;
    }
    if (t == INFLOW) continue;  // output independent of the input
    double f[27];
    int src_of[27];
    int64_t srcs[27];
    for (int i = 0; i < 27; ++i) {
      const int64_t src = g.pull_src(n, i);
      srcs[i] = src;
      if (type && type[src] == SOLID) {
        f[i] = reconstruct(opposite(i), mp[n], 0);
        src_of[i] = -1;
      } else {
        f[i] = reconstruct(i, mp[src], 0);
        src_of[i] = 1;
      }
    }
    double Fx[3];
    load_force(F, N, n, Fx);
    Mom<double> ob = load(lo.data(), N, n);
    double fb[27], Fbn[3] = {0, 0, 0};
    moments_vjp(f, Fx, ob, fb, Fbn);
    for (int a = 0; a < 3; ++a) Fb[3 * n + a] += Fbn[a];
    for (int i = 0; i < 27; ++i) {
      if (src_of[i] < 0)
        reconstruct_vjp(opposite(i), mp[n], fb[i], mpb[n], 0);
      else
        reconstruct_vjp(i, mp[srcs[i]], fb[i], mpb[srcs[i]], 0);
    }
  }
  // Pass 1 reversed: through the collision.
  for (int64_t n = 0; n < N; ++n) {
    const uint8_t t = type ? type[n] : FLUID;
    if (t == SOLID) continue;
    double Fx[3];
    load_force(F, N, n, Fx);
    Mom<double> mb = zero_mom();
    double Fbn[3] = {0, 0, 0};
    collide_vjp(load(m, N, n), Fx, tau, mpb[n], mb, Fbn);
    store(lam_in, N, n, mb);
    for (int a = 0; a < 3; ++a) Fb[3 * n + a] += Fbn[a];
  }
  if (gF)
    for (int64_t n = 0; n < N; ++n)
      for (int a = 0; a < 3; ++a) gF[a * N + n] += Fb[3 * n + a];
}

// FP64 mass and kinetic energy over non-solid cells.
void orc_reduce(int64_t N, const double* m, const uint8_t* type, double* mass, double* ke) {
  double M = 0.0, E = 0.0;
  for (int64_t n = 0; n < N; ++n) {
    if (type && type[n] == SOLID) continue;
    const double rho = m[n];
    const double u2 = m[N + n] * m[N + n] + m[2 * N + n] * m[2 * N + n] + m[3 * N + n] * m[3 * N + n];
    M += rho;
    E += 0.5 * rho * u2;
  }
  *mass = M;
  *ke = E;
}

// Dither values of one cell (for tests of the generator).
void orc_dither(uint32_t x, uint32_t y, uint32_t z, uint32_t t, uint32_t seed, float* d) {
  dither10(x, y, z, t, seed, d);
}

// Encode stored variables (FP32, component-major 10 x N; component 0 is
// rho - 1) into codes of b_ru / b_s bits.  deterministic != 0 uses d = 1/2 (round
// to nearest) for every component.
void orc_encode_bits(int nx, int ny, int nz, const float* v, uint32_t t, uint32_t seed,
                     int deterministic, int b_ru, int b_s, uint16_t* q) {
  Grid g{nx, ny, nz};
  const int64_t N = g.N();
  const Bits bits{b_ru, b_s};
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    float d[10];
    if (deterministic) {
      for (int k = 0; k < 10; ++k) d[k] = 0.5f;
    } else {
      const uint32_t x = uint32_t(n % nx), y = uint32_t((n / nx) % ny), z = uint32_t(n / (int64_t(nx) * ny));
      dither10(x, y, z, t, seed, d);
    }
    for (int k = 0; k < 10; ++k) q[k * N + n] = encode_one(v[k * N + n], k, d[k], bits);
  }
}
void orc_encode(int nx, int ny, int nz, const float* v, uint32_t t, uint32_t seed, int deterministic,
                uint16_t* q) {
  orc_encode_bits(nx, ny, nz, v, t, seed, deterministic, 16, 16, q);
}

// Mean code of the FP32 value mp (rho - 1 for k = 0) over every dither field
// value of component k (the expectation of the stochastic rounding).
double orc_mean_code_over_dither_bits(float mp, int k, int b_ru, int b_s) {
  const uint32_t n = 1u << dither_bits(k);
  double s = 0.0;
  for (uint32_t f = 0; f < n; ++f) s += encode_one(mp, k, dither_of_field(k, f), Bits{b_ru, b_s});
  return s / double(n);
}
double orc_mean_code_over_dither(float mp, int k) { return orc_mean_code_over_dither_bits(mp, k, 16, 16); }

// Exact code-space coordinate (m' - c)/step + qc of an FP32 value, in FP64.
double orc_code_coordinate_bits(float mp, int k, int b_ru, int b_s) {
  const QGroup g = qgroup(k, Bits{b_ru, b_s});
  return (double(mp) - (g.lo + g.qc * (g.hi - g.lo) / g.Q)) * g.Q / (g.hi - g.lo) + g.qc;
}
double orc_code_coordinate(float mp, int k) { return orc_code_coordinate_bits(mp, k, 16, 16); }

void orc_decode_bits(int64_t N, const uint16_t* q, int b_ru, int b_s, double* v) {
  const Bits bits{b_ru, b_s};
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n)
    for (int k = 0; k < 10; ++k) v[k * N + n] = decode_one(q[k * N + n], k, bits);
}
void orc_decode(int64_t N, const uint16_t* q, double* v) { orc_decode_bits(N, q, 16, 16, v); }

void orc_ranges(double* lo, double* hi) {
  for (int k = 0; k < 10; ++k) {
    lo[k] = QLO[k];
    hi[k] = QHI[k];
  }
}

// Grid constants of component k: centre code, FP32 step, FP32 value of the
// centre code (shifted variable), K and b of the encoding.
void orc_codec_constants_bits(int k, int b_ru, int b_s, double* out /*5*/) {
  const Bits bits{b_ru, b_s};
  out[0] = qgroup(k, bits).qc;
  out[1] = q_step(k, bits);
  out[2] = q_c(k, bits);
  out[3] = q_K(k, bits);
  out[4] = q_b(k, bits);
}
void orc_codec_constants(int k, double* out /*5*/) { orc_codec_constants_bits(k, 16, 16, out); }

}  // extern "C"
