// HWENO-I oracle: a plain, slow CPU implementation of the fifth-order finite-difference
// interpolation-based Hermite WENO scheme (Xie, Tao, Jiao, Zhang, arXiv 2411.11229).
//
// TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg of the
// benchmark are the only callers.  Nothing in the product library links or calls this file,
// and this file shares no code, header or constant table with the CUDA path.
//
// Everything is FP64 and is meant to be compiled with -ffp-contract=off (the `_ext` entry points
// run the same templated formulas in long double, as the reference that FP64 rounding is measured
// against).  Every formula is written in the order and notation of the paper:
//   Sec. 2, Eq. (EQ1)/(odeH)      augmented system and conservative semi-discretisation (1D)
//   Sec. 2.1, Eqs. (HWEp0)-(limiter)  Hermite candidates, smoothness indicators, weights,
//                                      interpolation and HWENO limiter
//   Sec. 2.2, Eqs. (Pc),(Cd-1),(DfDh) central Hermite correction D(f), D(h)
//   Eqs. (flux-1d),(flux-LF)      Lax-Friedrichs numerical fluxes
//   Eq. (fully-hweno), (2Dfully-hweno)  SSP-RK3 with the modified derivative in the base
//   Sec. 3, Eqs. (EQ3),(ode2H),(mixed)  2D system, dimension-by-dimension fluxes, mixed fluxes
//   Remarks after Sec. 2.2 and Sec. 3: local characteristic decomposition for Euler
//   Remarks (RBC-1d), (RBC-2d-x), (RBC-2d-y): reflective boundary tables
//
// Readings where the paper is silent (see the design notes of the repository):
//   * p0 has five conditions and is therefore degree 4 (the paper calls it quintic).
//   * u^+ at x_{i-1/2} is the mirror image of u^- at x_{i+1/2}: the same procedure applied to the
//     data reflected about x_i (derivatives change sign).  With gamma1 = gamma2 the weights are
//     then the same numbers as those of u^-.
//   * v^+/- is the linear p0' value (Eq. interp); the weights are shared by u^+/- and v~.
//   * alpha of the Lax-Friedrichs flux is one global maximum of |f'(u)| (Euler: |u|+c, |v|+c)
//     over the cells of the stage input, per direction, recomputed at every stage.
//   * Characteristic decomposition: at face i+1/2 the Roe average of U_i and U_{i+1} gives the
//     eigenvectors; all stencil values (solution and derivative) are projected with them.  The
//     modified derivative of cell i uses the eigenvectors of U_i.  D-terms, LF and mixed fluxes
//     are componentwise.
//   * Transmissive boundary: zero-order extrapolation of U and of its derivatives.
//   * Fixed-state side (the top and bottom of Example 4.11): the ghost cells hold the given state
//     with zero derivatives.
//   * Gravity source (Eq. euler2d-s, 2D Euler): L_U gains (0, 0, g rho, g rho nu); the derivative
//     equations gain its derivatives, g (0, 0, V_rho, V_rhonu) and g (0, 0, W_rho, W_rhonu), taken
//     from the stage input's own derivative fields (the semi-discrete operator; the modified
//     derivative enters only the base of the time step).
//   * dt = CFL dx / alpha (1D), CFL / (alpha_x/dx + alpha_y/dy) (2D); optional power p on dx.
//
// Variants (flags; the default is the scheme above):
//   FLAG_V_WEIGHTED  v^+/- combined with the nonlinear weights of u^+/- (the abstract's wording)
//                    instead of the linear p0' value.
//   FLAG_CD2         D-terms from Eq. (Cd-2) (h at the two inner nodes) instead of Eq. (Cd-1).
//   FLAG_R2          characteristic decomposition with the eigenvectors of the stencil's own
//                    centre cell (U_i for u^-_{i+1/2}, U_{i+1} for u^+_{i+1/2}) instead of the
//                    Roe average at the face.
//   FLAG_ALPHA_STEP  the LF coefficients of the first stage's input held for all three stages.
//   FLAG_ALPHA_LOCAL local LF (Rusanov): alpha at face i+1/2 is the larger spectral radius of the
//                    two adjacent cells i, i+1 (ghost cells through the boundary map).
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>
#include <algorithm>

namespace hwo {

// ---------------------------------------------------------------------------------------------
// Threads.  The operator is evaluated line by line (a row for the x sweep, a column for the y
// sweep) and cell by cell; every face flux, modified derivative and updated value is written by
// exactly one line or cell, and no value's arithmetic depends on which thread computes it or on
// the order in which lines are taken.  Splitting the lines (and the cell-wise loops) into
// contiguous chunks over threads therefore gives results that are bit for bit those of one thread.
inline int& thread_count() {
  static int n = 0;  // 0: all hardware threads
  return n;
}
inline int threads_used() {
  int n = thread_count();
  if (n <= 0) n = (int)std::thread::hardware_concurrency();
  return n < 1 ? 1 : n;
}
// body(lo, hi) on contiguous chunks of [0, n), one chunk per thread, each chunk at least `grain`
// long
template <class F>
void parallel_for(long long n, F body, long long grain = 1) {
  const long long T = std::min<long long>(threads_used(), n / std::max(1LL, grain));
  if (T <= 1) {
    if (n > 0) body(0LL, n);
    return;
  }
  const long long chunk = (n + T - 1) / T;
  std::vector<std::thread> th;
  for (long long lo = 0; lo < n; lo += chunk) th.emplace_back(body, lo, std::min(n, lo + chunk));
  for (auto& t : th) t.join();
}

using std::fabs;
using std::sqrt;

enum { ADVECTION = 0, BURGERS = 1, EULER = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_FIXED = 3 };
enum { FLAG_V_WEIGHTED = 1, FLAG_CD2 = 2, FLAG_R2 = 4, FLAG_ALPHA_STEP = 8, FLAG_ALPHA_LOCAL = 16 };

struct Cfg {
  int32_t dim, system, nx, ny, bc, flags;
  double dx, dy, gamma, gamma0, d0, eps, ax, ay;
  double grav;         // g of Eq. (euler2d-s); 0 = no source
  int32_t side[4];     // boundary type of the sides x-low, x-high, y-low, y-high
  double fixed[4][4];  // conserved state in the ghost cells of a BC_FIXED side
};

inline int ncomp(const Cfg& c) { return c.system == EULER ? (c.dim == 1 ? 3 : 4) : 1; }
inline int nfield(const Cfg& c) { return c.dim == 1 ? 2 : 3; }

template <class R> inline R sq(const R& a) { return a * a; }

// ---------------------------------------------------------------------------------------------
// Sec. 2.1: one HWENO stencil T0 = {i-1,i,i+1} with T1 = {i-1,i}, T2 = {i,i+1}.
// Inputs: u_{i-1}, u_i, u_{i+1}, v_{i-1}, v_{i+1}.  A face needs the value and derivative at
// x_{i+1/2} (u^-_{i+1/2}, v^-_{i+1/2}, Eq. interp, weights from gamma); a cell needs the modified
// derivative at x_i (Eq. limiter, weights from d).  Both share the smoothness indicators; the
// pieces below are combined per use, and hweno_stencil gives every intermediate for the unit tests.

// Eqs. (Pxi), (P'xi): p_l(x_{i+1/2}) and p0'(x_{i+1/2})
template <class R>
void face_candidates(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx, R p[3], R& dp0) {
  p[0] = -(1.0 / 8.0) * um + (9.0 / 16.0) * u0 + (9.0 / 16.0) * up - dx * ((3.0 / 64.0) * vm + (9.0 / 64.0) * vp);
  p[1] = -(1.0 / 2.0) * um + (3.0 / 2.0) * u0;
  p[2] = (1.0 / 2.0) * u0 + (1.0 / 2.0) * up;
  dp0 = (1.0 / dx) * ((3.0 / 16.0) * um - (3.0 / 2.0) * u0 + (21.0 / 16.0) * up) + (1.0 / 16.0) * vm - (3.0 / 16.0) * vp;
}

// the slopes p1', p2' of the two linear candidates (Eq. limiter-p)
template <class R>
void candidate_slopes(const R& um, const R& u0, const R& up, double dx, R& dp1, R& dp2) {
  dp1 = (1.0 / dx) * (u0 - um);
  dp2 = (1.0 / dx) * (up - u0);
}

// Eq. (limiter-p): p_l'(x_i)
template <class R>
void centre_derivatives(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx, R dpc[3]) {
  dpc[0] = (3.0 / (4.0 * dx)) * (up - um) - (1.0 / 4.0) * (vm + vp);
  candidate_slopes(um, u0, up, dx, dpc[1], dpc[2]);
}

// smoothness indicators (explicit form of Eq. GHYZ) and tau of Eq. (nonlinear)
template <class R>
void indicators(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx, R beta[3], R& tau) {
  R a1 = -(dx / 4.0) * (vm + vp) + (3.0 / 4.0) * (up - um);
  R a2 = (dx / 4.0) * (vm - vp) + (um - 2.0 * u0 + up);
  R a3 = (dx / 4.0) * (vm + vp) + (1.0 / 4.0) * (um - up);
  R a4 = (dx / 4.0) * (vp - vm) - (1.0 / 2.0) * (um - 2.0 * u0 + up);
  beta[0] = sq(a1 + (1.0 / 4.0) * a3) + (13.0 / 3.0) * sq(a2 + (63.0 / 130.0) * a4) + (781.0 / 20.0) * sq(a3) +
            (1421461.0 / 2275.0) * sq(a4);
  beta[1] = sq(u0 - um);
  beta[2] = sq(u0 - up);
  tau = (1.0 / 4.0) * sq(fabs(beta[0] - beta[1]) + fabs(beta[0] - beta[2]));
}

// Eq. (nonlinear): the weights omega_l from the linear weights lin (gamma or d)
template <class R>
void nonlinear_weights(const R beta[3], const R& tau, const double lin[3], double eps, R w[3]) {
  R wb[3];
  for (int l = 0; l < 3; ++l) wb[l] = lin[l] * (1.0 + tau / (beta[l] + eps));
  R s = wb[0] + wb[1] + wb[2];
  for (int l = 0; l < 3; ++l) w[l] = wb[l] / s;
}

// Eqs. (interp), (limiter): w0 (c0 / lin0 - (lin1 / lin0) c1 - (lin2 / lin0) c2) + w1 c1 + w2 c2
template <class R>
R combine(const R w[3], const double lin[3], const R c[3]) {
  return w[0] * ((1.0 / lin[0]) * c[0] - (lin[1] / lin[0]) * c[1] - (lin[2] / lin[0]) * c[2]) + w[1] * c[1] +
         w[2] * c[2];
}

// every intermediate of one stencil (unit tests)
template <class R>
struct StencilOut {
  R p[3];      // p_l(x_{i+1/2}), Eq. (Pxi)
  R dp0;       // p0'(x_{i+1/2}), Eq. (P'xi)
  R dpc[3];    // p_l'(x_i), Eq. (limiter-p)
  R beta[3];   // smoothness indicators
  R tau;
  R wg[3];     // omega^gamma
  R wd[3];     // omega^d
  R u_half;    // u^-_{i+1/2}
  R v_half;    // v^-_{i+1/2}
  R v_mod;     // v~_i
};

template <class R>
void hweno_stencil(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx,
                   const double g[3], const double d[3], double eps, StencilOut<R>& o, bool v_weighted = false) {
  face_candidates(um, u0, up, vm, vp, dx, o.p, o.dp0);
  centre_derivatives(um, u0, up, vm, vp, dx, o.dpc);
  indicators(um, u0, up, vm, vp, dx, o.beta, o.tau);
  nonlinear_weights(o.beta, o.tau, g, eps, o.wg);
  nonlinear_weights(o.beta, o.tau, d, eps, o.wd);
  o.u_half = combine(o.wg, g, o.p);
  o.v_half = o.dp0;
  if (v_weighted) {
    // the same combination applied to the derivatives at x_{i+1/2}; p1 and p2 are linear, so
    // their derivatives there are their slopes
    const R c[3] = {o.dp0, o.dpc[1], o.dpc[2]};
    o.v_half = combine(o.wg, g, c);
  }
  o.v_mod = combine(o.wd, d, o.dpc);
}

// u^-_{i+1/2}, v^-_{i+1/2} from the stencil of cell i (Eqs. Pxi, P'xi, GHYZ, nonlinear, interp).
template <class R>
void interp_minus(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx, const double g[3],
                  double eps, R& u_half, R& v_half, bool vw = false) {
  R beta[3], tau, w[3], p[3], dp0, c[3];
  face_candidates(um, u0, up, vm, vp, dx, p, dp0);
  if (vw) candidate_slopes(um, u0, up, dx, c[1], c[2]);
  indicators(um, u0, up, vm, vp, dx, beta, tau);
  nonlinear_weights(beta, tau, g, eps, w);
  u_half = combine(w, g, p);
  v_half = dp0;
  if (vw) {
    c[0] = dp0;
    v_half = combine(w, g, c);
  }
}

// u^+_{i-1/2}, v^+_{i-1/2} from the stencil of cell i: the mirror image of interp_minus.  The
// data are reflected about x_i (x -> 2 x_i - x): values swap ends, derivatives change sign.
template <class R>
void interp_plus(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx, const double g[3],
                 double eps, R& u_half, R& v_half, bool vw = false) {
  R nvp = -vp, nvm = -vm;
  interp_minus(up, u0, um, nvp, nvm, dx, g, eps, u_half, v_half, vw);
  v_half = -v_half;
}

// v~_i from the stencil of cell i (Eqs. limiter-p, GHYZ, nonlinear with d, limiter).
template <class R>
R limited_derivative(const R& um, const R& u0, const R& up, const R& vm, const R& vp, double dx, const double d[3],
                     double eps) {
  R beta[3], tau, w[3], dpc[3];
  centre_derivatives(um, u0, up, vm, vp, dx, dpc);
  indicators(um, u0, up, vm, vp, dx, beta, tau);
  nonlinear_weights(beta, tau, d, eps, w);
  return combine(w, d, dpc);
}

// ---------------------------------------------------------------------------------------------
// Sec. 2.2, Eqs. (Cd-1) and (DfDh): from f_{i-1..i+2} and h_{i-1}, h_{i+2}.
template <class R>
void dterms(const R& fm, const R& f0, const R& f1, const R& f2, const R& hm, const R& h2, double dx, R& Df, R& Dh) {
  R P2 = (9.0 / 8.0) * (fm - f0 - f1 + f2) + (5.0 / 12.0) * dx * (hm - h2);                 // dx^2 P''
  R P3 = -(1.0 / dx) * ((101.0 / 36.0) * fm - (27.0 / 4.0) * f0 + (27.0 / 4.0) * f1 - (101.0 / 36.0) * f2) -
         (5.0 / 6.0) * (hm + h2);                                                             // dx^2 P'''
  R P4 = -3.0 * (fm - f0 - f1 + f2) - 2.0 * dx * (hm - h2);                                  // dx^4 P''''
  R P5 = (1.0 / dx) * ((130.0 / 9.0) * fm - 30.0 * f0 + 30.0 * f1 - (130.0 / 9.0) * f2) +
         (20.0 / 3.0) * (hm + h2);                                                            // dx^4 P^(5)
  Df = -(1.0 / 24.0) * P2 + (7.0 / 5760.0) * P4;
  Dh = -(1.0 / 24.0) * P3 + (7.0 / 5760.0) * P5;
}

// The alternative of the remark after Eq. (D6): Eq. (Cd-2), from the Hermite interpolant (Pc2)
// of f_{i-1..i+2} and h_i, h_{i+1}, combined by Eq. (DfDh) as before.
template <class R>
void dterms2(const R& fm, const R& f0, const R& f1, const R& f2, const R& h0, const R& h1, double dx, R& Df, R& Dh) {
  R P2 = -(1.0 / 8.0) * (fm - f0 - f1 + f2) - (5.0 / 4.0) * dx * (h0 - h1);                  // dx^2 P''
  R P3 = (1.0 / (4.0 * dx)) * (fm + 57.0 * f0 - 57.0 * f1 - f2) + (15.0 / 2.0) * (h0 + h1);  // dx^2 P'''
  R P4 = 3.0 * (fm - f0 - f1 + f2) + 6.0 * dx * (h0 - h1);                                     // dx^4 P''''
  R P5 = -(10.0 / dx) * (fm + 9.0 * f0 - 9.0 * f1 - f2) - 60.0 * (h0 + h1);                    // dx^4 P^(5)
  Df = -(1.0 / 24.0) * P2 + (7.0 / 5760.0) * P4;
  Dh = -(1.0 / 24.0) * P3 + (7.0 / 5760.0) * P5;
}

// ---------------------------------------------------------------------------------------------
// Physical fluxes.  dir = 0 is x, dir = 1 is y.  Euler equations (euler1d)/(euler2d) with
// E = P/(gamma-1) + rho |mu|^2 / 2.
template <class R>
struct Phys {
  const Cfg& c;
  explicit Phys(const Cfg& cc) : c(cc) {}

  // f(u) or g(u): the physical flux of U in direction dir
  void flux(int dir, const R* U, R* F) const {
    if (c.system == ADVECTION) {
      F[0] = (dir == 0 ? c.ax : c.ay) * U[0];
    } else if (c.system == BURGERS) {
      F[0] = 0.5 * U[0] * U[0];
    } else if (c.dim == 1) {
      R rho = U[0], mu = U[1] / rho, E = U[2];
      R P = (c.gamma - 1.0) * (E - 0.5 * rho * mu * mu);
      F[0] = rho * mu;
      F[1] = rho * mu * mu + P;
      F[2] = mu * (E + P);
    } else {
      R rho = U[0], mu = U[1] / rho, nu = U[2] / rho, E = U[3];
      R P = (c.gamma - 1.0) * (E - 0.5 * rho * (mu * mu + nu * nu));
      if (dir == 0) {
        F[0] = rho * mu;
        F[1] = rho * mu * mu + P;
        F[2] = rho * mu * nu;
        F[3] = mu * (E + P);
      } else {
        F[0] = rho * nu;
        F[1] = rho * mu * nu;
        F[2] = rho * nu * nu + P;
        F[3] = nu * (E + P);
      }
    }
  }

  // Flux Jacobian dF_dir/dU as an explicit matrix (textbook form, H = (E+P)/rho).
  void jacobian(int dir, const R* U, R* A /* m x m, row major */) const {
    int m = ncomp(c);
    if (c.system == ADVECTION) {
      A[0] = R(dir == 0 ? c.ax : c.ay);
      return;
    }
    if (c.system == BURGERS) {
      A[0] = U[0];
      return;
    }
    double gm = c.gamma - 1.0;
    if (c.dim == 1) {
      R rho = U[0], u = U[1] / rho, E = U[2];
      R P = gm * (E - 0.5 * rho * u * u);
      R H = (E + P) / rho;
      R Arow[9] = {R(0.0), R(1.0), R(0.0),
                   0.5 * (c.gamma - 3.0) * u * u, (3.0 - c.gamma) * u, R(gm),
                   u * (0.5 * gm * u * u - H), H - gm * u * u, c.gamma * u};
      for (int k = 0; k < 9; ++k) A[k] = Arow[k];
      (void)m;
      return;
    }
    R rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
    R q2 = u * u + v * v;
    R P = gm * (E - 0.5 * rho * q2);
    R H = (E + P) / rho;
    if (dir == 0) {
      R Arow[16] = {R(0.0), R(1.0), R(0.0), R(0.0),
                    0.5 * gm * q2 - u * u, (3.0 - c.gamma) * u, -gm * v, R(gm),
                    -u * v, v, u, R(0.0),
                    u * (0.5 * gm * q2 - H), H - gm * u * u, -gm * u * v, c.gamma * u};
      for (int k = 0; k < 16; ++k) A[k] = Arow[k];
    } else {
      R Arow[16] = {R(0.0), R(0.0), R(1.0), R(0.0),
                    -u * v, v, u, R(0.0),
                    0.5 * gm * q2 - v * v, -gm * u, (3.0 - c.gamma) * v, R(gm),
                    v * (0.5 * gm * q2 - H), -gm * u * v, H - gm * v * v, c.gamma * v};
      for (int k = 0; k < 16; ++k) A[k] = Arow[k];
    }
  }

  // h = f'(u) v (Eq. EQ1) and its 2D relatives xi, eta, theta (Eq. EQ3): Jacobian times a
  // derivative vector.
  void jac_vec(int dir, const R* U, const R* V, R* out) const {
    int m = ncomp(c);
    R A[16];
    jacobian(dir, U, A);
    for (int r = 0; r < m; ++r) {
      R s = A[r * m] * V[0];
      for (int k = 1; k < m; ++k) s = s + A[r * m + k] * V[k];
      out[r] = s;
    }
  }

  // |f'(u)| (scalar) or the spectral radius |velocity| + c (Euler) at one cell
  R wavespeed(int dir, const R* U) const {
    if (c.system == ADVECTION) return R(fabs(dir == 0 ? c.ax : c.ay));
    if (c.system == BURGERS) return fabs(U[0]);
    if (c.dim == 1) {
      R rho = U[0], u = U[1] / rho, E = U[2];
      R P = (c.gamma - 1.0) * (E - 0.5 * rho * u * u);
      return fabs(u) + sqrt(c.gamma * P / rho);
    }
    R rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
    R P = (c.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    return fabs(dir == 0 ? u : v) + sqrt(c.gamma * P / rho);
  }
};

// ---------------------------------------------------------------------------------------------
// Local characteristic decomposition (Euler).  The averaged state (u, v, H, c) and the textbook
// right eigenvectors of the direction-dir Jacobian, ordered by eigenvalue (vel-c, vel, [shear],
// vel+c).  L is the closed-form inverse of R.
template <class R>
struct EigenState {
  R u, v, H, c;
};

template <class R>
EigenState<R> roe_average(const Cfg& cf, const R* UL, const R* UR) {
  double gm = cf.gamma - 1.0;
  EigenState<R> s;
  if (cf.dim == 1) {
    R rl = UL[0], ul = UL[1] / rl, El = UL[2];
    R rr = UR[0], ur = UR[1] / rr, Er = UR[2];
    R Pl = gm * (El - 0.5 * rl * ul * ul), Pr = gm * (Er - 0.5 * rr * ur * ur);
    R Hl = (El + Pl) / rl, Hr = (Er + Pr) / rr;
    R sl = sqrt(rl), sr = sqrt(rr);
    s.u = (sl * ul + sr * ur) / (sl + sr);
    s.v = R(0.0);
    s.H = (sl * Hl + sr * Hr) / (sl + sr);
    s.c = sqrt(gm * (s.H - 0.5 * s.u * s.u));
    return s;
  }
  R rl = UL[0], ul = UL[1] / rl, vl = UL[2] / rl, El = UL[3];
  R rr = UR[0], ur = UR[1] / rr, vr = UR[2] / rr, Er = UR[3];
  R Pl = gm * (El - 0.5 * rl * (ul * ul + vl * vl)), Pr = gm * (Er - 0.5 * rr * (ur * ur + vr * vr));
  R Hl = (El + Pl) / rl, Hr = (Er + Pr) / rr;
  R sl = sqrt(rl), sr = sqrt(rr);
  s.u = (sl * ul + sr * ur) / (sl + sr);
  s.v = (sl * vl + sr * vr) / (sl + sr);
  s.H = (sl * Hl + sr * Hr) / (sl + sr);
  s.c = sqrt(gm * (s.H - 0.5 * (s.u * s.u + s.v * s.v)));
  return s;
}

// eigen-state of one cell: the local state itself
template <class R>
EigenState<R> cell_state(const Cfg& cf, const R* U) {
  double gm = cf.gamma - 1.0;
  EigenState<R> s;
  if (cf.dim == 1) {
    R rho = U[0], u = U[1] / rho, E = U[2];
    R P = gm * (E - 0.5 * rho * u * u);
    s.u = u;
    s.v = R(0.0);
    s.H = (E + P) / rho;
    s.c = sqrt(cf.gamma * P / rho);
    return s;
  }
  R rho = U[0], u = U[1] / rho, v = U[2] / rho, E = U[3];
  R P = gm * (E - 0.5 * rho * (u * u + v * v));
  s.u = u;
  s.v = v;
  s.H = (E + P) / rho;
  s.c = sqrt(cf.gamma * P / rho);
  return s;
}

// Right eigenvectors as the columns of Rm (row-major m x m).
template <class R>
void right_eigen(const Cfg& cf, int dir, const EigenState<R>& s, R* Rm) {
  const R &u = s.u, &v = s.v, &H = s.H, &c = s.c;
  if (cf.dim == 1) {
    R K[3][3] = {{R(1.0), u - c, H - u * c}, {R(1.0), u, 0.5 * u * u}, {R(1.0), u + c, H + u * c}};
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) Rm[r * 3 + k] = K[k][r];
    return;
  }
  R q = 0.5 * (u * u + v * v);
  if (dir == 0) {
    R K[4][4] = {{R(1.0), u - c, v, H - u * c}, {R(1.0), u, v, q}, {R(0.0), R(0.0), R(1.0), v}, {R(1.0), u + c, v, H + u * c}};
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) Rm[r * 4 + k] = K[k][r];
  } else {
    R K[4][4] = {{R(1.0), u, v - c, H - v * c}, {R(1.0), u, v, q}, {R(0.0), R(1.0), R(0.0), u}, {R(1.0), u, v + c, H + v * c}};
    for (int r = 0; r < 4; ++r)
      for (int k = 0; k < 4; ++k) Rm[r * 4 + k] = K[k][r];
  }
}

// Left eigenvectors (rows of Lm), the inverse of right_eigen, with b1 = (gamma-1)/c^2 and
// b2 = b1 |vel|^2 / 2.
template <class R>
void left_eigen(const Cfg& cf, int dir, const EigenState<R>& s, R* Lm) {
  double gm = cf.gamma - 1.0;
  const R &u = s.u, &v = s.v, &c = s.c;
  R b1 = gm / (c * c);
  if (cf.dim == 1) {
    R b2 = 0.5 * b1 * u * u;
    R L[9] = {0.5 * (b2 + u / c), -0.5 * (b1 * u + 1.0 / c), 0.5 * b1,
              1.0 - b2, b1 * u, -b1,
              0.5 * (b2 - u / c), -0.5 * (b1 * u - 1.0 / c), 0.5 * b1};
    for (int k = 0; k < 9; ++k) Lm[k] = L[k];
    return;
  }
  R b2 = 0.5 * b1 * (u * u + v * v);
  if (dir == 0) {
    R L[16] = {0.5 * (b2 + u / c), -0.5 * (b1 * u + 1.0 / c), -0.5 * b1 * v, 0.5 * b1,
               1.0 - b2, b1 * u, b1 * v, -b1,
               -v, R(0.0), R(1.0), R(0.0),
               0.5 * (b2 - u / c), -0.5 * (b1 * u - 1.0 / c), -0.5 * b1 * v, 0.5 * b1};
    for (int k = 0; k < 16; ++k) Lm[k] = L[k];
  } else {
    R L[16] = {0.5 * (b2 + v / c), -0.5 * b1 * u, -0.5 * (b1 * v + 1.0 / c), 0.5 * b1,
               1.0 - b2, b1 * u, b1 * v, -b1,
               -u, R(1.0), R(0.0), R(0.0),
               0.5 * (b2 - v / c), -0.5 * b1 * u, -0.5 * (b1 * v - 1.0 / c), 0.5 * b1};
    for (int k = 0; k < 16; ++k) Lm[k] = L[k];
  }
}

template <class R>
void matvec(int m, const R* M, const R* x, R* y) {
  for (int r = 0; r < m; ++r) {
    R s = M[r * m] * x[0];
    for (int k = 1; k < m; ++k) s = s + M[r * m + k] * x[k];
    y[r] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// Ghost-padded copy of a state.  Layout of a state: [field][comp][ny][nx], x fastest.
// Fields: 1D (U, V), 2D (U, V, W) with V = U_x and W = U_y.
template <class R>
struct Padded {
  int nf, nc, nx, ny, gx, gy, px, py;
  std::vector<R> a;
  Padded(const Cfg& c)
      : nf(nfield(c)), nc(ncomp(c)), nx(c.nx), ny(c.dim == 2 ? c.ny : 1), gx(2), gy(c.dim == 2 ? 2 : 0) {
    px = nx + 2 * gx;
    py = ny + 2 * gy;
    a.assign((size_t)nf * nc * px * py, R(0.0));
  }
  R& at(int f, int k, int j, int i) { return a[(((size_t)f * nc + k) * py + (j + gy)) * px + (i + gx)]; }
  const R& at(int f, int k, int j, int i) const { return a[(((size_t)f * nc + k) * py + (j + gy)) * px + (i + gx)]; }
};

// Sign of a reflected ghost value (Remarks RBC-1d, RBC-2d-x, RBC-2d-y): wall normal to dir.
inline double reflect_sign(const Cfg& c, int dir, int field, int comp) {
  if (c.dim == 1) {
    static const double U[3] = {1, -1, 1}, V[3] = {-1, 1, -1};
    return field == 0 ? U[comp] : V[comp];
  }
  // rows: U, V = U_x, W = U_y; columns: rho, rho mu, rho nu, E
  static const double X[3][4] = {{1, -1, 1, 1}, {-1, 1, -1, -1}, {1, -1, 1, 1}};
  static const double Y[3][4] = {{1, 1, -1, 1}, {1, 1, -1, 1}, {-1, -1, 1, -1}};
  return dir == 0 ? X[field][comp] : Y[field][comp];
}

// index of the interior cell that supplies ghost/interior index i on an axis of n cells, for a
// side of type bc (periodic, transmissive or reflective)
inline int bc_source(int bc, int i, int n, bool* flipped) {
  *flipped = false;
  if (i >= 0 && i < n) return i;
  if (bc == BC_PERIODIC) return ((i % n) + n) % n;
  if (bc == BC_TRANSMISSIVE) return i < 0 ? 0 : n - 1;
  *flipped = true;  // reflective: mirror about the wall
  return i < 0 ? -1 - i : 2 * n - 1 - i;
}

// Where the value of field f, component k at cell (j, i) (interior or ghost) comes from: either
// sgn * S[idx], or the constant `value` (a fixed-state side).
struct Source {
  bool fixed;
  double value, sgn;
  size_t idx;
};

inline Source boundary_source(const Cfg& c, int f, int k, int j, int i) {
  const int m = ncomp(c);
  const int nx = c.nx, ny = c.dim == 2 ? c.ny : 1;
  Source s{false, 0.0, 1.0, 0};
  int si = i, sj = j;
  const int sx = i < 0 ? 0 : (i >= nx ? 1 : -1);
  const int sy = c.dim == 1 ? -1 : (j < 0 ? 2 : (j >= ny ? 3 : -1));
  for (int side : {sx, sy}) {
    if (side < 0) continue;
    if (c.side[side] == BC_FIXED) {
      s.fixed = true;
      s.value = f == 0 ? c.fixed[side][k] : 0.0;  // the state, with zero derivatives
      return s;
    }
  }
  bool fx = false, fy = false;
  if (sx >= 0) si = bc_source(c.side[sx], i, nx, &fx);
  if (sy >= 0) sj = bc_source(c.side[sy], j, ny, &fy);
  if (fx) s.sgn *= reflect_sign(c, 0, f, k);
  if (fy) s.sgn *= reflect_sign(c, 1, f, k);
  s.idx = ((size_t)f * m + k) * ((size_t)nx * ny) + (size_t)sj * nx + si;
  return s;
}

template <class R>
R boundary_value(const Cfg& c, const R* S, int f, int k, int j, int i) {
  const Source s = boundary_source(c, f, k, j, i);
  if (s.fixed) return R(s.value);
  return s.sgn == 1.0 ? S[s.idx] : -S[s.idx];
}

template <class R>
void fill_padded(const Cfg& c, const R* S, Padded<R>& P) {
  const long long rows = (long long)P.nf * P.nc * P.py;  // padded rows (f, k, j)
  parallel_for(rows, [&](long long lo, long long hi) {
    for (long long r = lo; r < hi; ++r) {
      const int j = (int)(r % P.py) - P.gy, k = (int)((r / P.py) % P.nc), f = (int)(r / ((long long)P.py * P.nc));
      for (int i = -P.gx; i < P.nx + P.gx; ++i) P.at(f, k, j, i) = boundary_value(c, S, f, k, j, i);
    }
  }, std::max(1, (1 << 14) / P.px));
}

// ---------------------------------------------------------------------------------------------
// The stage operator.  Given the stage input S, produce L(S) (Eq. odeH / ode2H, all fields) and
// M(S) = (U, V~, W~): the solution and the modified derivatives (Eq. limiter) that enter the
// SSP-RK3 update (Eq. fully-hweno / 2Dfully-hweno).  alpha_x, alpha_y: the LF coefficients.
template <class R>
struct Operator {
  const Cfg& c;
  Phys<R> ph;
  int m, nf;
  double g[3], d[3];
  Operator(const Cfg& cc) : c(cc), ph(cc), m(ncomp(cc)), nf(nfield(cc)) {
    g[0] = c.gamma0;
    g[1] = g[2] = 0.5 * (1.0 - c.gamma0);
    d[0] = c.d0;
    d[1] = d[2] = 0.5 * (1.0 - c.d0);
  }

  // Step (1.1)/(2.1) for one face and direction: U and D (D = V for x, W for y) of the four
  // cells k-1..k+2 around face k+1/2 -> U^-, D^-, U^+, D^+ at the face.
  void face_states(int dir, R Uc[4][4], R Dc[4][4], R* Um, R* Dm, R* Up, R* Dp) const {
    double h = dir == 0 ? c.dx : c.dy;
    const bool vw = (c.flags & FLAG_V_WEIGHTED) != 0;
    if (c.system != EULER) {
      interp_minus(Uc[0][0], Uc[1][0], Uc[2][0], Dc[0][0], Dc[2][0], h, g, c.eps, Um[0], Dm[0], vw);
      interp_plus(Uc[1][0], Uc[2][0], Uc[3][0], Dc[1][0], Dc[3][0], h, g, c.eps, Up[0], Dp[0], vw);
      return;
    }
    // local characteristic decomposition: one basis at the face (Roe average), or with FLAG_R2
    // the basis of each side's centre cell (U_k for the minus side, U_{k+1} for the plus side)
    const bool r2 = (c.flags & FLAG_R2) != 0;
    EigenState<R> sm = r2 ? cell_state(c, Uc[1]) : roe_average(c, Uc[1], Uc[2]);
    EigenState<R> sp = r2 ? cell_state(c, Uc[2]) : sm;
    R Rmm[16], Lmm[16], Rpp[16], Lpp[16];
    right_eigen(c, dir, sm, Rmm);
    left_eigen(c, dir, sm, Lmm);
    if (r2) {
      right_eigen(c, dir, sp, Rpp);
      left_eigen(c, dir, sp, Lpp);
    } else {
      for (int e = 0; e < 16; ++e) {
        Rpp[e] = Rmm[e];
        Lpp[e] = Lmm[e];
      }
    }
    R Wm[4][4], Zm[4][4], Wp[4][4], Zp[4][4];
    for (int q = 0; q < 4; ++q) {
      matvec(m, Lmm, Uc[q], Wm[q]);
      matvec(m, Lmm, Dc[q], Zm[q]);
      for (int k = 0; k < m; ++k) {
        Wp[q][k] = Wm[q][k];
        Zp[q][k] = Zm[q][k];
      }
      if (r2) {
        matvec(m, Lpp, Uc[q], Wp[q]);
        matvec(m, Lpp, Dc[q], Zp[q]);
      }
    }
    R wm[4], zm[4], wp[4], zp[4];
    for (int s2 = 0; s2 < m; ++s2) {
      interp_minus(Wm[0][s2], Wm[1][s2], Wm[2][s2], Zm[0][s2], Zm[2][s2], h, g, c.eps, wm[s2], zm[s2], vw);
      interp_plus(Wp[1][s2], Wp[2][s2], Wp[3][s2], Zp[1][s2], Zp[3][s2], h, g, c.eps, wp[s2], zp[s2], vw);
    }
    matvec(m, Rmm, wm, Um);
    matvec(m, Rmm, zm, Dm);
    matvec(m, Rpp, wp, Up);
    matvec(m, Rpp, zp, Dp);
  }

  // modified derivative of one cell from U, D of cells i-1, i, i+1 (Eq. limiter)
  void modified_derivative(int dir, R Uc[3][4], R Dc[3][4], R* Dt) const {
    double h = dir == 0 ? c.dx : c.dy;
    if (c.system != EULER) {
      Dt[0] = limited_derivative(Uc[0][0], Uc[1][0], Uc[2][0], Dc[0][0], Dc[2][0], h, d, c.eps);
      return;
    }
    EigenState<R> s = cell_state(c, Uc[1]);
    R Rm[16], Lm[16];
    right_eigen(c, dir, s, Rm);
    left_eigen(c, dir, s, Lm);
    R W[3][4], Z[3][4];
    for (int q = 0; q < 3; ++q) {
      matvec(m, Lm, Uc[q], W[q]);
      matvec(m, Lm, Dc[q], Z[q]);
    }
    R zt[4];
    for (int s2 = 0; s2 < m; ++s2) zt[s2] = limited_derivative(W[0][s2], W[1][s2], W[2][s2], Z[0][s2], Z[2][s2], h, d, c.eps);
    matvec(m, Rm, zt, Dt);
  }

  // the largest wavespeed over the cells (a maximum is exact, so splitting the cells over threads
  // gives the same value)
  R max_wavespeed(int dir, const R* S) const {
    const int ny = c.dim == 2 ? c.ny : 1;
    const size_t plane = (size_t)c.nx * ny;
    R a = R(0.0);
    std::mutex mu;
    parallel_for((long long)plane, [&](long long lo, long long hi) {
      R am = R(0.0);
      for (size_t p = (size_t)lo; p < (size_t)hi; ++p) {
        R U[4];
        for (int k = 0; k < m; ++k) U[k] = S[k * plane + p];
        R w = ph.wavespeed(dir, U);
        if (w > am) am = w;
      }
      std::lock_guard<std::mutex> lock(mu);
      if (am > a) a = am;
    }, 1 << 15);
    return a;
  }

  // Steps (1.1)-(1.3) / (2.1)-(2.3) and Step 3 for one face k+1/2 in direction dir, from the four
  // cells k-1..k+2: U, the derivative field of this direction D (V for x, W for y) and, in 2D,
  // the other derivative field O.  Outputs the flux of U (f^ or g^), of D (h^ or theta^) and
  // the mixed flux of O (eta^ or xi^).
  void face_flux(int dir, R Uc[4][4], R Dc[4][4], R Oc[4][4], R alpha, R* fhat, R* hhat, R* mixed) const {
    double h = dir == 0 ? c.dx : c.dy;
    if (c.flags & FLAG_ALPHA_LOCAL) {
      const R al = ph.wavespeed(dir, Uc[1]), ar = ph.wavespeed(dir, Uc[2]);
      alpha = ar > al ? ar : al;
    }
    // Step 1.1: interface values
    R Um[4], Dm[4], Up[4], Dp[4];
    face_states(dir, Uc, Dc, Um, Dm, Up, Dp);
    // nodal fluxes for the D-terms (Eq. Pc: f at k-1..k+2, h at k-1 and k+2; Eq. Pc2: h at k, k+1)
    R fn[4][4], hn[4][4], on[4][4];
    for (int q = 0; q < 4; ++q) {
      ph.flux(dir, Uc[q], fn[q]);
      ph.jac_vec(dir, Uc[q], Dc[q], hn[q]);
      if (c.dim == 2) ph.jac_vec(dir, Uc[q], Oc[q], on[q]);
    }
    // Step 1.3: Eqs. (flux-1d), (flux-LF)
    R FUm[4], FUp[4], HDm[4], HDp[4];
    ph.flux(dir, Um, FUm);
    ph.flux(dir, Up, FUp);
    ph.jac_vec(dir, Um, Dm, HDm);
    ph.jac_vec(dir, Up, Dp, HDp);
    for (int k = 0; k < m; ++k) {
      R Df, Dh;
      if (c.flags & FLAG_CD2)
        dterms2(fn[0][k], fn[1][k], fn[2][k], fn[3][k], hn[1][k], hn[2][k], h, Df, Dh);
      else
        dterms(fn[0][k], fn[1][k], fn[2][k], fn[3][k], hn[0][k], hn[3][k], h, Df, Dh);
      fhat[k] = 0.5 * (FUm[k] + FUp[k] - alpha * (Up[k] - Um[k])) + Df;
      hhat[k] = 0.5 * (HDm[k] + HDp[k] - alpha * (Dp[k] - Dm[k])) + Dh;
      if (c.dim == 2) {
        // Eq. (mixed): linear fourth-order flux of the other derivative field
        mixed[k] = -(1.0 / 12.0) * on[0][k] + (7.0 / 12.0) * on[1][k] + (7.0 / 12.0) * on[2][k] -
                   (1.0 / 12.0) * on[3][k];
      }
    }
  }

  // L and M of one stage.  alpha: the LF coefficients (x, y).
  void rhs(const R* S, R* Lout, R* Mout, R alpha_x, R alpha_y) const {
    Padded<R> P(c);
    fill_padded(c, S, P);
    const int nx = c.nx, ny = c.dim == 2 ? c.ny : 1;
    const size_t plane = (size_t)nx * ny;
    const int nfl = nf;  // fields
    // face fluxes: x faces (nx+1 per row), y faces (ny+1 per column); [field][comp][...]
    std::vector<R> FX((size_t)nfl * m * ny * (nx + 1), R(0.0));
    std::vector<R> FY(c.dim == 2 ? (size_t)nfl * m * (ny + 1) * nx : 0, R(0.0));
    auto fx = [&](int f, int k, int j, int i) -> R& { return FX[(((size_t)f * m + k) * ny + j) * (nx + 1) + i]; };
    auto fy = [&](int f, int k, int j, int i) -> R& { return FY[(((size_t)f * m + k) * (ny + 1) + j) * nx + i]; };

    for (int dir = 0; dir < c.dim; ++dir) {
      const R alpha = dir == 0 ? alpha_x : alpha_y;
      const int own = dir == 0 ? 1 : 2;    // derivative field interpolated in this direction
      const int other = dir == 0 ? 2 : 1;  // derivative field with the mixed flux (2D)
      const int nlines = dir == 0 ? ny : nx;
      const int nalong = dir == 0 ? nx : ny;
      // lines are independent: each writes only its own faces and cells
      parallel_for(nlines, [&](long long line_lo, long long line_hi) {
      for (int line = (int)line_lo; line < (int)line_hi; ++line) {
        auto cellF = [&](int f, int a, R* D) {
          for (int k = 0; k < m; ++k) D[k] = dir == 0 ? P.at(f, k, line, a) : P.at(f, k, a, line);
        };
        // faces a+1/2, a = -1 .. nalong-1
        for (int a = -1; a < nalong; ++a) {
          R Uc[4][4], Dc[4][4], Oc[4][4];
          for (int q = 0; q < 4; ++q) {
            cellF(0, a - 1 + q, Uc[q]);
            cellF(own, a - 1 + q, Dc[q]);
            if (c.dim == 2) cellF(other, a - 1 + q, Oc[q]);
          }
          R fh[4], hh[4], mx[4];
          face_flux(dir, Uc, Dc, Oc, alpha, fh, hh, mx);
          for (int k = 0; k < m; ++k) {
            if (dir == 0) {
              fx(0, k, line, a + 1) = fh[k];
              fx(own, k, line, a + 1) = hh[k];
              if (c.dim == 2) fx(other, k, line, a + 1) = mx[k];
            } else {
              fy(0, k, a + 1, line) = fh[k];
              fy(own, k, a + 1, line) = hh[k];
              fy(other, k, a + 1, line) = mx[k];
            }
          }
        }
        // modified derivative of every cell on the line
        for (int a = 0; a < nalong; ++a) {
          R Uc[3][4], Dc[3][4], Dt[4];
          for (int q = 0; q < 3; ++q) {
            cellF(0, a - 1 + q, Uc[q]);
            cellF(own, a - 1 + q, Dc[q]);
          }
          modified_derivative(dir, Uc, Dc, Dt);
          for (int k = 0; k < m; ++k) {
            size_t p = dir == 0 ? (size_t)line * nx + a : (size_t)a * nx + line;
            Mout[((size_t)own * m + k) * plane + p] = Dt[k];
          }
        }
      }
      });
    }
    // Step 4: the conservative differences (row by row)
    parallel_for((long long)nfl * m * ny, [&](long long lo, long long hi) {
      for (long long r = lo; r < hi; ++r) {
        const int j = (int)(r % ny), k = (int)((r / ny) % m), f = (int)(r / ((long long)ny * m));
        for (int i = 0; i < nx; ++i) {
          R val = -(1.0 / c.dx) * (fx(f, k, j, i + 1) - fx(f, k, j, i));
          if (c.dim == 2) val = val - (1.0 / c.dy) * (fy(f, k, j + 1, i) - fy(f, k, j, i));
          Lout[((size_t)f * m + k) * plane + (size_t)j * nx + i] = val;
        }
      }
    }, std::max(1, (1 << 14) / nx));
    if (c.grav != 0.0)
      for (int f = 0; f < nfl; ++f)
        for (size_t p = 0; p < plane; ++p) {
          R src[4];
          source(f, [&](int k) { return S[((size_t)f * m + k) * plane + p]; }, src);
          for (int k = 0; k < m; ++k) Lout[((size_t)f * m + k) * plane + p] = Lout[((size_t)f * m + k) * plane + p] + src[k];
        }
    for (int k = 0; k < m; ++k)
      for (size_t p = 0; p < plane; ++p) Mout[(size_t)k * plane + p] = S[(size_t)k * plane + p];
  }

  // Eq. (euler2d-s): the gravity source of field f (U: g (0, 0, rho, rho nu); a derivative field:
  // the same expression in that field's components), with val(k) the cell's component k of field f.
  template <class Get>
  void source(int f, Get val, R* src) const {
    (void)f;
    for (int k = 0; k < m; ++k) src[k] = R(0.0);
    if (c.grav == 0.0) return;
    src[2] = c.grav * val(0);
    src[3] = c.grav * val(2);
  }

  // The same L and M at selected cells only, reading S through the boundary map (for checks at
  // sizes where the full operator is too slow on the CPU).  Lout, Mout: [ncell][field][comp].
  void rhs_cells(const R* S, R alpha_x, R alpha_y, long long ncell, const long long* idx, R* Lout, R* Mout) const {
    const int nx = c.nx, ny = c.dim == 2 ? c.ny : 1;
    const size_t plane = (size_t)nx * ny;
    (void)plane;
    auto value = [&](int f, int k, int j, int i) -> R { return boundary_value(c, S, f, k, j, i); };
    for (long long s = 0; s < ncell; ++s) {
      const int i = (int)(idx[s] % nx), j = (int)(idx[s] / nx);
      R Lc[3][4], Mc[3][4];
      for (int f = 0; f < nf; ++f)
        for (int k = 0; k < m; ++k) Lc[f][k] = R(0.0);
      for (int k = 0; k < m; ++k) Mc[0][k] = value(0, k, j, i);
      for (int dir = 0; dir < c.dim; ++dir) {
        const R alpha = dir == 0 ? alpha_x : alpha_y;
        const int own = dir == 0 ? 1 : 2, other = dir == 0 ? 2 : 1;
        const double inv_h = dir == 0 ? 1.0 / c.dx : 1.0 / c.dy;
        auto at = [&](int f, int k, int off) -> R { return dir == 0 ? value(f, k, j, i + off) : value(f, k, j + off, i); };
        R fl[2][3][4];  // faces -1/2 and +1/2: [face][field][comp]
        for (int side = 0; side < 2; ++side) {
          R Uc[4][4], Dc[4][4], Oc[4][4];
          for (int q = 0; q < 4; ++q)
            for (int k = 0; k < m; ++k) {
              int off = side - 2 + q;  // face i-1/2: cells i-2..i+1; face i+1/2: i-1..i+2
              Uc[q][k] = at(0, k, off);
              Dc[q][k] = at(own, k, off);
              Oc[q][k] = c.dim == 2 ? at(other, k, off) : R(0.0);
            }
          R fh[4], hh[4], mx[4];
          face_flux(dir, Uc, Dc, Oc, alpha, fh, hh, mx);
          for (int k = 0; k < m; ++k) {
            fl[side][0][k] = fh[k];
            fl[side][own][k] = hh[k];
            if (c.dim == 2) fl[side][other][k] = mx[k];
          }
        }
        for (int f = 0; f < nf; ++f)
          for (int k = 0; k < m; ++k) Lc[f][k] = Lc[f][k] - inv_h * (fl[1][f][k] - fl[0][f][k]);
        R Uc[3][4], Dc[3][4], Dt[4];
        for (int q = 0; q < 3; ++q)
          for (int k = 0; k < m; ++k) {
            Uc[q][k] = at(0, k, q - 1);
            Dc[q][k] = at(own, k, q - 1);
          }
        modified_derivative(dir, Uc, Dc, Dt);
        for (int k = 0; k < m; ++k) Mc[own][k] = Dt[k];
      }
      if (c.grav != 0.0)
        for (int f = 0; f < nf; ++f) {
          R src[4];
          source(f, [&](int k) { return value(f, k, j, i); }, src);
          for (int k = 0; k < m; ++k) Lc[f][k] = Lc[f][k] + src[k];
        }
      for (int f = 0; f < nf; ++f)
        for (int k = 0; k < m; ++k) {
          Lout[((size_t)s * nf + f) * m + k] = Lc[f][k];
          Mout[((size_t)s * nf + f) * m + k] = Mc[f][k];
        }
    }
  }
};

// Stage st of Eq. (fully-hweno) / (2Dfully-hweno) from L and M of the stage input: at the first
// stage B = M(S^n) (u^n and the modified derivatives) and S = M + dt L; then
// S = a_k B + b_k (M + dt L) with (a_k, b_k) = (3/4, 1/4), (1/3, 2/3).  Value by value.
template <class R>
void rk3_combine(int st, size_t n, double dt, const R* L, const R* M, R* B, R* S) {
  static const double a_k[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0};
  static const double b_k[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};
  parallel_for((long long)n, [&](long long lo, long long hi) {
    for (long long p = lo; p < hi; ++p) {
      if (st == 0) {
        B[p] = M[p];
        S[p] = M[p] + dt * L[p];
      } else {
        S[p] = a_k[st] * B[p] + b_k[st] * (M[p] + dt * L[p]);
      }
    }
  }, 1 << 15);
}

// One SSP-RK3 step with the modified derivative in the base (Eq. fully-hweno / 2Dfully-hweno).
// S is updated in place.  alpha per stage from the stage input.
template <class R>
void rk3_step(const Cfg& c, R* S, double dt) {
  Operator<R> op(c);
  const int ny = c.dim == 2 ? c.ny : 1;
  const size_t n = (size_t)nfield(c) * ncomp(c) * c.nx * ny;
  std::vector<R> L(n), M(n), B(n);
  R ax0 = R(0.0), ay0 = R(0.0);
  for (int st = 0; st < 3; ++st) {
    R ax = op.max_wavespeed(0, S);
    R ay = c.dim == 2 ? op.max_wavespeed(1, S) : R(0.0);
    if (c.flags & FLAG_ALPHA_STEP) {
      if (st == 0) {
        ax0 = ax;
        ay0 = ay;
      }
      ax = ax0;
      ay = ay0;
    }
    op.rhs(S, L.data(), M.data(), ax, ay);
    rk3_combine(st, n, dt, L.data(), M.data(), B.data(), S);
  }
}

template <class R>
double cfl_dt(const Cfg& c, const R* S, double cfl, double dx_pow) {
  Operator<R> op(c);
  double ax = (double)op.max_wavespeed(0, S);
  if (c.dim == 1) return cfl * std::pow(c.dx, dx_pow) / ax;
  double ay = (double)op.max_wavespeed(1, S);
  return cfl / (ax / std::pow(c.dx, dx_pow) + ay / std::pow(c.dy, dx_pow));
}

// ---------------------------------------------------------------------------------------------
// Operation counting: the same templated code instantiated with a scalar that counts every
// floating-point +, -, *, / and sqrt applied to the data.  A Counted is either a value computed
// from the data (made by Counted::data) or a constant of the scheme (a literal or a parameter,
// what every implicit conversion from double makes).  Not counted: sign changes, fabs and
// comparisons; operations between constants (the constant folding any implementation does once);
// and operations with a structural constant 0 or +-1: a product with such a factor, a quotient by
// +-1 or of 0, a sum with a term 0.  These are the zeros and ones of the explicit Jacobian and
// eigenvector matrices, which a plain matrix-vector product multiplies and adds like any other
// entry, and the zero initial values of sums.  Values of the data are counted whatever they are,
// so the counts do not depend on the data (the arithmetic has no data-dependent branches).
struct Counted {
  double v;
  bool k;  // a constant of the scheme, not a value computed from the data
  Counted() : v(0.0), k(true) {}
  Counted(double x) : v(x), k(true) {}
  static Counted data(double x) {
    Counted c(x);
    c.k = false;
    return c;
  }
  static Counted make(double x, bool konst) {
    Counted c(x);
    c.k = konst;
    return c;
  }
  static long long& n() {
    static long long c = 0;
    return c;
  }
};
inline bool const0(const Counted& a) { return a.k && a.v == 0.0; }
inline bool const1(const Counted& a) { return a.k && (a.v == 1.0 || a.v == -1.0); }
inline Counted operator+(const Counted& a, const Counted& b) {
  if (!(a.k && b.k) && !const0(a) && !const0(b)) ++Counted::n();
  return Counted::make(a.v + b.v, a.k && b.k);
}
inline Counted operator-(const Counted& a, const Counted& b) {
  if (!(a.k && b.k) && !const0(a) && !const0(b)) ++Counted::n();
  return Counted::make(a.v - b.v, a.k && b.k);
}
inline Counted operator*(const Counted& a, const Counted& b) {
  const bool zero = const0(a) || const0(b);
  if (!(a.k && b.k) && !zero && !const1(a) && !const1(b)) ++Counted::n();
  return Counted::make(a.v * b.v, (a.k && b.k) || zero);
}
inline Counted operator/(const Counted& a, const Counted& b) {
  if (!(a.k && b.k) && !const0(a) && !const1(b)) ++Counted::n();
  return Counted::make(a.v / b.v, (a.k && b.k) || const0(a));
}
inline Counted operator-(const Counted& a) { return Counted::make(-a.v, a.k); }
inline bool operator>(const Counted& a, const Counted& b) { return a.v > b.v; }
inline Counted fabs(const Counted& a) { return Counted::make(std::fabs(a.v), a.k); }
inline Counted sqrt(const Counted& a) {
  if (!a.k) ++Counted::n();
  return Counted::make(std::sqrt(a.v), a.k);
}

// ---------------------------------------------------------------------------------------------
// Derivatives of the scheme for the adjoint (conventions: the step sizes and the LF coefficients
// alpha of every stage are held fixed at recorded values; d|x|/dx = sign(x) with sign(0) = 0).
//
// Reverse mode: `Adj` records every operation on a tape (two parents with their partial
// derivatives); one reverse sweep gives the gradient of a weighted sum of outputs.  The tape is
// kept per face or per cell (the operator is local), so its size stays small.
// Forward mode: `Dual` carries one directional derivative through the same code.
struct Tape {
  std::vector<int> a, b;
  std::vector<double> da, db;
  void clear() {
    a.clear();
    b.clear();
    da.clear();
    db.clear();
  }
  int push(int ia, double pa, int ib, double pb) {
    a.push_back(ia);
    b.push_back(ib);
    da.push_back(pa);
    db.push_back(pb);
    return (int)a.size() - 1;
  }
  size_t size() const { return a.size(); }
};
inline Tape& tape() {
  static thread_local Tape t;
  return t;
}

struct Adj {
  double v;
  int id;  // tape index, -1 for a constant
  Adj() : v(0.0), id(-1) {}
  Adj(double x) : v(x), id(-1) {}
  Adj(double x, int i) : v(x), id(i) {}
};
inline Adj adj_var(double x) { return Adj(x, tape().push(-1, 0.0, -1, 0.0)); }
inline Adj adj_node(double v, int ia, double pa, int ib, double pb) {
  if (ia < 0 && ib < 0) return Adj(v);
  return Adj(v, tape().push(ia, pa, ib, pb));
}
inline Adj operator+(const Adj& x, const Adj& y) { return adj_node(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline Adj operator-(const Adj& x, const Adj& y) { return adj_node(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline Adj operator*(const Adj& x, const Adj& y) { return adj_node(x.v * y.v, x.id, y.v, y.id, x.v); }
inline Adj operator/(const Adj& x, const Adj& y) {
  const double q = x.v / y.v;
  return adj_node(q, x.id, 1.0 / y.v, y.id, -q / y.v);
}
inline Adj operator-(const Adj& x) { return adj_node(-x.v, x.id, -1.0, -1, 0.0); }
inline bool operator>(const Adj& x, const Adj& y) { return x.v > y.v; }
inline Adj fabs(const Adj& x) { return adj_node(std::fabs(x.v), x.id, x.v > 0 ? 1.0 : (x.v < 0 ? -1.0 : 0.0), -1, 0.0); }
inline Adj sqrt(const Adj& x) {
  const double r = std::sqrt(x.v);
  return adj_node(r, x.id, 0.5 / r, -1, 0.0);
}

// reverse sweep: adjoint of every tape entry from the seeds already placed in g
inline void adj_sweep(std::vector<double>& g) {
  const Tape& t = tape();
  for (int i = (int)t.size() - 1; i >= 0; --i) {
    const double gi = g[i];
    if (gi == 0.0) continue;
    if (t.a[i] >= 0) g[t.a[i]] += t.da[i] * gi;
    if (t.b[i] >= 0) g[t.b[i]] += t.db[i] * gi;
  }
}

struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double y) : v(x), d(y) {}
};
inline Dual operator+(const Dual& x, const Dual& y) { return Dual(x.v + y.v, x.d + y.d); }
inline Dual operator-(const Dual& x, const Dual& y) { return Dual(x.v - y.v, x.d - y.d); }
inline Dual operator*(const Dual& x, const Dual& y) { return Dual(x.v * y.v, x.d * y.v + x.v * y.d); }
inline Dual operator/(const Dual& x, const Dual& y) {
  const double q = x.v / y.v;
  return Dual(q, (x.d - q * y.d) / y.v);
}
inline Dual operator-(const Dual& x) { return Dual(-x.v, -x.d); }
inline bool operator>(const Dual& x, const Dual& y) { return x.v > y.v; }
inline Dual fabs(const Dual& x) { return Dual(std::fabs(x.v), x.v > 0 ? x.d : (x.v < 0 ? -x.d : 0.0)); }
inline Dual sqrt(const Dual& x) {
  const double r = std::sqrt(x.v);
  return Dual(r, 0.5 * x.d / r);
}

// Vector-Jacobian product of one stage operator at S with alpha fixed:
// lam = (dM/dS)^T muM + (dL/dS)^T muL (all arrays in the state layout).
inline void stage_vjp(const Cfg& c, const double* S, double ax, double ay, const double* muM, const double* muL,
                      double* lam) {
  Operator<Adj> op(c);
  const int m = ncomp(c), nf = nfield(c);
  const int nx = c.nx, ny = c.dim == 2 ? c.ny : 1;
  const size_t plane = (size_t)nx * ny;
  const size_t n = (size_t)nf * m * plane;
  for (size_t p = 0; p < n; ++p) lam[p] = 0.0;
  for (int k = 0; k < m; ++k)
    for (size_t p = 0; p < plane; ++p) lam[k * plane + p] += muM[k * plane + p];  // M = (U, ...)
  // boundary map of a cell (f, k, j, i) to its source cell and sign
  // (a fixed-state ghost value is a constant: sign 0, so it receives no adjoint)
  auto source = [&](int f, int k, int j, int i, size_t* idx, double* val) -> double {
    const Source s = boundary_source(c, f, k, j, i);
    if (s.fixed) {
      *idx = 0;
      *val = s.value;
      return 0.0;
    }
    *idx = s.idx;
    *val = s.sgn * S[s.idx];
    return s.sgn;
  };
  double vu = 0.0, vd = 0.0, vo = 0.0;
  // the gravity source is linear in S: L_f[2] += g S_f[0], L_f[3] += g S_f[2]
  if (c.grav != 0.0)
    for (int f = 0; f < nf; ++f)
      for (size_t p = 0; p < plane; ++p) {
        lam[((size_t)f * m + 0) * plane + p] += c.grav * muL[((size_t)f * m + 2) * plane + p];
        lam[((size_t)f * m + 2) * plane + p] += c.grav * muL[((size_t)f * m + 3) * plane + p];
      }
  std::vector<double> g;
  for (int dir = 0; dir < c.dim; ++dir) {
    const double h = dir == 0 ? c.dx : c.dy;
    const double alpha = dir == 0 ? ax : ay;
    const int own = dir == 0 ? 1 : 2, other = dir == 0 ? 2 : 1;
    const int nlines = dir == 0 ? ny : nx, nalong = dir == 0 ? nx : ny;
    for (int line = 0; line < nlines; ++line) {
      auto cell = [&](int a, int* jj, int* ii) {
        *jj = dir == 0 ? line : a;
        *ii = dir == 0 ? a : line;
      };
      auto mu_at = [&](const double* mu, int f, int k, int a) -> double {
        if (a < 0 || a >= nalong) return 0.0;
        int jj, ii;
        cell(a, &jj, &ii);
        return mu[((size_t)f * m + k) * plane + (size_t)jj * nx + ii];
      };
      // faces a+1/2: the fluxes enter L of cells a (-1/h) and a+1 (+1/h)
      for (int a = -1; a < nalong; ++a) {
        tape().clear();
        Adj Uc[4][4], Dc[4][4], Oc[4][4];
        size_t iu[4][4], id[4][4], io[4][4];
        double su[4][4], sd[4][4], so[4][4];
        for (int q = 0; q < 4; ++q) {
          int jj, ii;
          cell(a - 1 + q, &jj, &ii);
          for (int k = 0; k < m; ++k) {
            su[q][k] = source(0, k, jj, ii, &iu[q][k], &vu);
            sd[q][k] = source(own, k, jj, ii, &id[q][k], &vd);
            Uc[q][k] = adj_var(vu);
            Dc[q][k] = adj_var(vd);
            if (c.dim == 2) {
              so[q][k] = source(other, k, jj, ii, &io[q][k], &vo);
              Oc[q][k] = adj_var(vo);
            }
          }
        }
        Adj fh[4], hh[4], mx[4];
        op.face_flux(dir, Uc, Dc, Oc, Adj(alpha), fh, hh, mx);
        g.assign(tape().size(), 0.0);
        for (int k = 0; k < m; ++k) {
          auto nu = [&](int f) { return (mu_at(muL, f, k, a + 1) - mu_at(muL, f, k, a)) / h; };
          if (fh[k].id >= 0) g[fh[k].id] += nu(0);
          if (hh[k].id >= 0) g[hh[k].id] += nu(own);
          if (c.dim == 2 && mx[k].id >= 0) g[mx[k].id] += nu(other);
        }
        adj_sweep(g);
        for (int q = 0; q < 4; ++q)
          for (int k = 0; k < m; ++k) {
            lam[iu[q][k]] += su[q][k] * g[Uc[q][k].id];
            lam[id[q][k]] += sd[q][k] * g[Dc[q][k].id];
            if (c.dim == 2) lam[io[q][k]] += so[q][k] * g[Oc[q][k].id];
          }
      }
      // modified derivative of every cell on the line
      for (int a = 0; a < nalong; ++a) {
        tape().clear();
        Adj Uc[3][4], Dc[3][4], Dt[4];
        size_t iu[3][4], id[3][4];
        double su[3][4], sd[3][4];
        for (int q = 0; q < 3; ++q) {
          int jj, ii;
          cell(a - 1 + q, &jj, &ii);
          for (int k = 0; k < m; ++k) {
            su[q][k] = source(0, k, jj, ii, &iu[q][k], &vu);
            sd[q][k] = source(own, k, jj, ii, &id[q][k], &vd);
            Uc[q][k] = adj_var(vu);
            Dc[q][k] = adj_var(vd);
          }
        }
        op.modified_derivative(dir, Uc, Dc, Dt);
        g.assign(tape().size(), 0.0);
        for (int k = 0; k < m; ++k)
          if (Dt[k].id >= 0) g[Dt[k].id] += mu_at(muM, own, k, a);
        adj_sweep(g);
        for (int q = 0; q < 3; ++q)
          for (int k = 0; k < m; ++k) {
            lam[iu[q][k]] += su[q][k] * g[Uc[q][k].id];
            lam[id[q][k]] += sd[q][k] * g[Dc[q][k].id];
          }
      }
    }
  }
  tape().clear();
}

// Jacobian-vector products of one stage operator at S along delta with alpha fixed.
inline void stage_jvp(const Cfg& c, const double* S, double ax, double ay, const double* delta, double* jM,
                      double* jL) {
  Operator<Dual> op(c);
  const int ny = c.dim == 2 ? c.ny : 1;
  const size_t n = (size_t)nfield(c) * ncomp(c) * c.nx * ny;
  std::vector<Dual> Sd(n), L(n), M(n);
  for (size_t p = 0; p < n; ++p) Sd[p] = Dual(S[p], delta[p]);
  op.rhs(Sd.data(), L.data(), M.data(), Dual(ax), Dual(ay));
  for (size_t p = 0; p < n; ++p) {
    jM[p] = M[p].d;
    jL[p] = L[p].d;
  }
}

// One SSP-RK3 step with given step size and given LF coefficients per stage
// (alpha6 = {ax, ay} of stages 1, 2, 3).
template <class R>
void rk3_step_alpha(const Cfg& c, R* S, double dt, const double* alpha6) {
  Operator<R> op(c);
  const int ny = c.dim == 2 ? c.ny : 1;
  const size_t n = (size_t)nfield(c) * ncomp(c) * c.nx * ny;
  std::vector<R> L(n), M(n), B(n);
  for (int st = 0; st < 3; ++st) {
    op.rhs(S, L.data(), M.data(), R(alpha6[2 * st]), R(alpha6[2 * st + 1]));
    rk3_combine(st, n, dt, L.data(), M.data(), B.data(), S);
  }
}

// Adjoint of one SSP-RK3 step (fixed dt, alpha6 as above): lam_out = (dS^{n+1}/dS^n)^T lam_in.
inline void adjoint_step(const Cfg& c, const double* Sn, double dt, const double* alpha6, const double* lam_in,
                         double* lam_out) {
  Operator<double> op(c);
  const int ny = c.dim == 2 ? c.ny : 1;
  const size_t n = (size_t)nfield(c) * ncomp(c) * c.nx * ny;
  std::vector<double> L(n), M(n), B(n), S1(n), S2(n);
  // forward stages, keeping the stage inputs
  op.rhs(Sn, L.data(), M.data(), alpha6[0], alpha6[1]);
  for (size_t p = 0; p < n; ++p) {
    B[p] = M[p];
    S1[p] = M[p] + dt * L[p];
  }
  op.rhs(S1.data(), L.data(), M.data(), alpha6[2], alpha6[3]);
  for (size_t p = 0; p < n; ++p) S2[p] = (3.0 / 4.0) * B[p] + (1.0 / 4.0) * (M[p] + dt * L[p]);
  // S^{n+1} = 1/3 B + 2/3 (M(S2) + dt L(S2))
  std::vector<double> muM(n), muL(n), lam2(n), lam1(n), lamB(n);
  for (size_t p = 0; p < n; ++p) {
    muM[p] = (2.0 / 3.0) * lam_in[p];
    muL[p] = (2.0 / 3.0) * dt * lam_in[p];
    lamB[p] = (1.0 / 3.0) * lam_in[p];
  }
  stage_vjp(c, S2.data(), alpha6[4], alpha6[5], muM.data(), muL.data(), lam2.data());
  // S2 = 3/4 B + 1/4 (M(S1) + dt L(S1))
  for (size_t p = 0; p < n; ++p) {
    muM[p] = (1.0 / 4.0) * lam2[p];
    muL[p] = (1.0 / 4.0) * dt * lam2[p];
    lamB[p] += (3.0 / 4.0) * lam2[p];
  }
  stage_vjp(c, S1.data(), alpha6[2], alpha6[3], muM.data(), muL.data(), lam1.data());
  // S1 = M(S^n) + dt L(S^n), B = M(S^n)
  for (size_t p = 0; p < n; ++p) {
    muM[p] = lam1[p] + lamB[p];
    muL[p] = dt * lam1[p];
  }
  stage_vjp(c, Sn, alpha6[0], alpha6[1], muM.data(), muL.data(), lam_out);
}

}  // namespace hwo

// =============================================================================================
// C interface (doubles only).  Return 0 on success, -1 on invalid arguments.
extern "C" {

typedef hwo::Cfg oracle_cfg;

static int check_cfg(const oracle_cfg* c) {
  if (!c) return -1;
  if (c->dim != 1 && c->dim != 2) return -1;
  if (c->system < 0 || c->system > 2) return -1;
  if (c->nx < 5 || (c->dim == 2 && c->ny < 5)) return -1;
  if (!(c->dx > 0) || (c->dim == 2 && !(c->dy > 0))) return -1;
  if (c->system == hwo::EULER && !(c->gamma > 1.0)) return -1;
  for (int sd = 0; sd < (c->dim == 2 ? 4 : 2); ++sd) {
    if (c->side[sd] < 0 || c->side[sd] > hwo::BC_FIXED) return -1;
    if (c->side[sd] == hwo::BC_REFLECTIVE && c->system != hwo::EULER) return -1;
  }
  // periodic pairs opposite sides
  if ((c->side[0] == hwo::BC_PERIODIC) != (c->side[1] == hwo::BC_PERIODIC)) return -1;
  if (c->dim == 2 && (c->side[2] == hwo::BC_PERIODIC) != (c->side[3] == hwo::BC_PERIODIC)) return -1;
  if (c->grav != 0.0 && !(c->dim == 2 && c->system == hwo::EULER)) return -1;  // Eq. (euler2d-s) only
  if (c->flags < 0 || c->flags > 31) return -1;
  if (!(c->gamma0 > 0 && c->gamma0 < 1) || !(c->d0 > 0 && c->d0 < 1) || !(c->eps > 0)) return -1;
  return 0;
}

// Threads of the operator (0: all hardware threads, the default; 1: serial).  The results do not
// depend on it (bit for bit).  Returns the number of threads the next calls use.
int oracle_set_threads(int n) {
  hwo::thread_count() = n < 0 ? 0 : n;
  return hwo::threads_used();
}

// number of doubles in one state
long long oracle_state_size(const oracle_cfg* c) {
  if (check_cfg(c)) return -1;
  return (long long)hwo::nfield(*c) * hwo::ncomp(*c) * c->nx * (c->dim == 2 ? c->ny : 1);
}

int oracle_max_wavespeed(const oracle_cfg* c, const double* S, double* ax, double* ay) {
  if (check_cfg(c)) return -1;
  hwo::Operator<double> op(*c);
  *ax = op.max_wavespeed(0, S);
  *ay = c->dim == 2 ? op.max_wavespeed(1, S) : 0.0;
  return 0;
}

// L(S) and M(S) = (U, V~, W~) with the LF coefficients taken from S
int oracle_rhs(const oracle_cfg* c, const double* S, double* L, double* M) {
  if (check_cfg(c)) return -1;
  hwo::Operator<double> op(*c);
  double ax = op.max_wavespeed(0, S);
  double ay = c->dim == 2 ? op.max_wavespeed(1, S) : 0.0;
  op.rhs(S, L, M, ax, ay);
  return 0;
}

// same with given LF coefficients
int oracle_rhs_alpha(const oracle_cfg* c, const double* S, double ax, double ay, double* L, double* M) {
  if (check_cfg(c)) return -1;
  hwo::Operator<double> op(*c);
  op.rhs(S, L, M, ax, ay);
  return 0;
}

// L and M at selected cells (flat indices j*nx+i) with given LF coefficients.
// Lout, Mout: [ncell][field][comp].
int oracle_rhs_cells(const oracle_cfg* c, const double* S, double ax, double ay, long long ncell,
                     const long long* idx, double* Lout, double* Mout) {
  if (check_cfg(c) || ncell < 0) return -1;
  hwo::Operator<double> op(*c);
  op.rhs_cells(S, ax, ay, ncell, idx, Lout, Mout);
  return 0;
}

// nsteps SSP-RK3 steps in place with a fixed dt
int oracle_steps(const oracle_cfg* c, double* S, double dt, int nsteps) {
  if (check_cfg(c) || nsteps < 0) return -1;
  for (int s = 0; s < nsteps; ++s) hwo::rk3_step(*c, S, dt);
  return 0;
}

// CFL dt of a state: cfl dx^p / alpha (1D) or cfl / (ax/dx^p + ay/dy^p) (2D)
double oracle_cfl_dt(const oracle_cfg* c, const double* S, double cfl, double dx_pow) {
  if (check_cfg(c)) return -1.0;
  return hwo::cfl_dt(*c, S, cfl, dx_pow);
}

// Run to t_end with CFL steps (last step clamped), or at most max_steps steps when t_end <= 0.
// Returns the number of steps taken, or -1.  *t_out = final time.
long long oracle_run(const oracle_cfg* c, double* S, double t_end, double cfl, double dx_pow, long long max_steps,
                     double* t_out) {
  if (check_cfg(c)) return -1;
  double t = 0.0;
  long long n = 0;
  while ((t_end <= 0.0 || t < t_end) && (max_steps <= 0 || n < max_steps)) {
    double dt = hwo::cfl_dt(*c, S, cfl, dx_pow);
    if (!(dt > 0) || !std::isfinite(dt)) return -1;
    if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    hwo::rk3_step(*c, S, dt);
    t += dt;
    ++n;
    if (t_end > 0.0 && t >= t_end) break;
  }
  if (t_out) *t_out = t;
  return n;
}

// Floating-point operation counts of the scheme as written (counting scalar):
// out[0] one face: interface values, fluxes at U^+-, D-terms, LF and mixed fluxes (the nodal
//        values of the four cells excluded);
// out[1] nodal values of one cell in one direction (f, f'(u) v and, in 2D, the mixed nodal value);
// out[2] modified derivative of one cell in one direction;  out[3] wavespeed of one cell, one
// direction;  out[4] conservative difference and SSP-RK3 combination of one cell (stage 2 form);
// out[5] one full SSP-RK3 step per cell: 3 (dim (faces + nodal + modified + wavespeed) + update).
int oracle_count_flops(const oracle_cfg* c, long long* out) {
  if (check_cfg(c)) return -1;
  using hwo::Counted;
  // spacings and speeds that are neither 0 nor +-1 (a parameter equal to 1 would make its products
  // structural)
  oracle_cfg cc = *c;
  cc.dx = 0.0371;
  cc.dy = 0.0293;
  cc.ax = 0.713;
  cc.ay = -0.537;
  hwo::Operator<Counted> op(cc);
  const int m = hwo::ncomp(cc);
  const int dim = cc.dim;
  long long& n = Counted::n();
  // four cells of a physical state (rho, momenta, E) with derivative data
  Counted Uc[4][4], Dc[4][4], Oc[4][4];
  for (int q = 0; q < 4; ++q)
    for (int k = 0; k < 4; ++k) {
      const double qq = 0.0419 * q * q;
      const double mom = k == 1 ? 0.2317 * q - 0.1109 - qq : -0.1931 + 0.0713 * q + qq;
      Uc[q][k] = Counted::data(k == 0 ? 1.3127 + 0.1713 * q + qq : (k == m - 1 ? 2.7139 + 0.1327 * q - qq : mom));
      Dc[q][k] = Counted::data(0.3137 * q - 0.2291 * k + 0.0517 + 0.0293 * q * q);
      Oc[q][k] = Counted::data(0.1123 * k - 0.2017 * q + 0.0331 - 0.0371 * q * q);
    }
  Counted fh[4], hh[4], mx[4];
  n = 0;
  op.face_flux(0, Uc, Dc, Oc, Counted::data(2.0317), fh, hh, mx);  // alpha: the data's wavespeed
  long long face_all = n;
  n = 0;
  Counted fn[4], hn[4], on[4];
  op.ph.flux(0, Uc[0], fn);
  op.ph.jac_vec(0, Uc[0], Dc[0], hn);
  if (dim == 2) op.ph.jac_vec(0, Uc[0], Oc[0], on);
  long long nodal = n;
  n = 0;
  Counted U3[3][4], D3[3][4], Dt[4];
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < 4; ++k) {
      U3[q][k] = Uc[q][k];
      D3[q][k] = Dc[q][k];
    }
  op.modified_derivative(0, U3, D3, Dt);
  long long md = n;
  n = 0;
  op.ph.wavespeed(0, Uc[0]);
  long long ws = n;
  // conservative difference (dim differences, each a subtraction and a scaling, summed) and the
  // stage combination a B + b (M + dt L) per value
  const long long nvals = (long long)hwo::nfield(cc) * m;
  long long upd = nvals * (dim == 2 ? 5 : 2) + nvals * 4;
  out[0] = face_all - 4 * nodal;
  out[1] = nodal;
  out[2] = md;
  out[3] = ws;
  out[4] = upd;
  out[5] = 3 * (dim * (out[0] + out[1] + out[2] + out[3]) + upd);
  n = 0;
  return 0;
}

// Operation counts (the convention of oracle_count_flops) of one scalar stencil of Sec. 2.1:
// out[0] the face part, u^- and v^- at x_{i+1/2} (Eqs. Pxi, P'xi, GHYZ, nonlinear with gamma,
// interp); out[1] the same with the weighted derivative of the FLAG_V_WEIGHTED variant;
// out[2] the cell part, v~_i (Eqs. limiter-p, GHYZ, nonlinear with d, limiter).
int oracle_count_stencil(long long* out) {
  using hwo::Counted;
  const double g[3] = {0.95, 0.025, 0.025}, d[3] = {0.9, 0.05, 0.05};
  const Counted um = Counted::data(1.3127), u0 = Counted::data(1.4841), up = Counted::data(1.2291);
  const Counted vm = Counted::data(0.3137), vp = Counted::data(-0.2019);
  long long& n = Counted::n();
  Counted a, b;
  n = 0;
  hwo::interp_minus(um, u0, up, vm, vp, 0.0371, g, 1e-10, a, b, false);
  out[0] = n;
  n = 0;
  hwo::interp_minus(um, u0, up, vm, vp, 0.0371, g, 1e-10, a, b, true);
  out[1] = n;
  n = 0;
  a = hwo::limited_derivative(um, u0, up, vm, vp, 0.0371, d, 1e-10);
  out[2] = n;
  n = 0;
  return 0;
}

// ---- extended precision ----
// The same templated formulas instantiated with long double (the x87 80-bit format, 64-bit
// significand, on x86-64; IEEE binary128, 113-bit significand, on AArch64): the state is read
// from double once, every value computed from the data is held and rounded in long double, and
// the results are rounded to double once at the end.  The coefficients of the scheme stay the
// double constants written above (literals, parameters, g, d, 1/h, dt), so this is the FP64
// oracle's arithmetic with its coefficients and with less rounding: the measure of how far an
// FP64 evaluation (the oracle's or the GPU's) is from the exact value of the same formulas.

int oracle_ext_mantissa_bits(void) { return LDBL_MANT_DIG; }

static std::vector<long double> to_ext(const double* S, size_t n) {
  std::vector<long double> v(n);
  for (size_t p = 0; p < n; ++p) v[p] = S[p];
  return v;
}

static size_t state_len(const oracle_cfg* c) {
  return (size_t)hwo::nfield(*c) * hwo::ncomp(*c) * c->nx * (c->dim == 2 ? c->ny : 1);
}

// L(S) and M(S) with the LF coefficients taken from S, all in long double
int oracle_rhs_ext(const oracle_cfg* c, const double* S, double* L, double* M) {
  if (check_cfg(c)) return -1;
  const size_t n = state_len(c);
  const std::vector<long double> Se = to_ext(S, n);
  std::vector<long double> Le(n), Me(n);
  hwo::Operator<long double> op(*c);
  const long double ax = op.max_wavespeed(0, Se.data());
  const long double ay = c->dim == 2 ? op.max_wavespeed(1, Se.data()) : 0.0L;
  op.rhs(Se.data(), Le.data(), Me.data(), ax, ay);
  for (size_t p = 0; p < n; ++p) {
    L[p] = (double)Le[p];
    M[p] = (double)Me[p];
  }
  return 0;
}

// L and M at selected cells (flat indices j*nx+i), the LF coefficients from the whole of S, all in
// long double.  Lout, Mout: [ncell][field][comp].
int oracle_rhs_cells_ext(const oracle_cfg* c, const double* S, long long ncell, const long long* idx, double* Lout,
                         double* Mout) {
  if (check_cfg(c) || ncell < 0) return -1;
  const size_t n = state_len(c);
  const std::vector<long double> Se = to_ext(S, n);
  hwo::Operator<long double> op(*c);
  const long double ax = op.max_wavespeed(0, Se.data());
  const long double ay = c->dim == 2 ? op.max_wavespeed(1, Se.data()) : 0.0L;
  const size_t nout = (size_t)ncell * hwo::nfield(*c) * hwo::ncomp(*c);
  std::vector<long double> Le(nout), Me(nout);
  const size_t per = (size_t)hwo::nfield(*c) * hwo::ncomp(*c);
  hwo::parallel_for(ncell, [&](long long lo, long long hi) {
    op.rhs_cells(Se.data(), ax, ay, hi - lo, idx + lo, Le.data() + (size_t)lo * per, Me.data() + (size_t)lo * per);
  });
  for (size_t p = 0; p < nout; ++p) {
    Lout[p] = (double)Le[p];
    Mout[p] = (double)Me[p];
  }
  return 0;
}

// Run to t_end with CFL steps (last step clamped), or at most max_steps steps when t_end <= 0, with
// the state held in long double between steps (each step's dt is a double, as in oracle_run).
long long oracle_run_ext(const oracle_cfg* c, double* S, double t_end, double cfl, double dx_pow,
                         long long max_steps, double* t_out) {
  if (check_cfg(c)) return -1;
  const size_t n = state_len(c);
  std::vector<long double> Se = to_ext(S, n);
  double t = 0.0;
  long long k = 0;
  while ((t_end <= 0.0 || t < t_end) && (max_steps <= 0 || k < max_steps)) {
    double dt = hwo::cfl_dt(*c, Se.data(), cfl, dx_pow);
    if (!(dt > 0) || !std::isfinite(dt)) return -1;
    if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    hwo::rk3_step(*c, Se.data(), dt);
    t += dt;
    ++k;
    if (t_end > 0.0 && t >= t_end) break;
  }
  for (size_t p = 0; p < n; ++p) S[p] = (double)Se[p];
  if (t_out) *t_out = t;
  return k;
}

// ---- derivatives (adjoint conventions: fixed dt and alpha per stage) ----

int oracle_stage_vjp(const oracle_cfg* c, const double* S, double ax, double ay, const double* muM,
                     const double* muL, double* lam) {
  if (check_cfg(c)) return -1;
  hwo::stage_vjp(*c, S, ax, ay, muM, muL, lam);
  return 0;
}

int oracle_stage_jvp(const oracle_cfg* c, const double* S, double ax, double ay, const double* delta, double* jM,
                     double* jL) {
  if (check_cfg(c)) return -1;
  hwo::stage_jvp(*c, S, ax, ay, delta, jM, jL);
  return 0;
}

// nsteps CFL steps recording dt (dts[nsteps]) and alpha of every stage (alphas[nsteps][6])
int oracle_steps_record(const oracle_cfg* c, double* S, int nsteps, double cfl, double* dts, double* alphas) {
  if (check_cfg(c) || nsteps < 0) return -1;
  hwo::Operator<double> op(*c);
  const int ny = c->dim == 2 ? c->ny : 1;
  const size_t n = (size_t)hwo::nfield(*c) * hwo::ncomp(*c) * c->nx * ny;
  std::vector<double> L(n), M(n), B(n);
  for (int s = 0; s < nsteps; ++s) {
    const double dt = hwo::cfl_dt(*c, S, cfl, 1.0);
    dts[s] = dt;
    for (int st = 0; st < 3; ++st) {
      const bool held = (c->flags & hwo::FLAG_ALPHA_STEP) && st > 0;
      const double ax = held ? alphas[6 * s] : op.max_wavespeed(0, S);
      const double ay = held ? alphas[6 * s + 1] : (c->dim == 2 ? op.max_wavespeed(1, S) : 0.0);
      alphas[6 * s + 2 * st] = ax;
      alphas[6 * s + 2 * st + 1] = ay;
      op.rhs(S, L.data(), M.data(), ax, ay);
      hwo::rk3_combine(st, n, dt, L.data(), M.data(), B.data(), S);
    }
  }
  return 0;
}

// nsteps steps with the recorded dts and alphas
int oracle_steps_replay(const oracle_cfg* c, double* S, int nsteps, const double* dts, const double* alphas) {
  if (check_cfg(c) || nsteps < 0) return -1;
  for (int s = 0; s < nsteps; ++s) hwo::rk3_step_alpha(*c, S, dts[s], alphas + 6 * s);
  return 0;
}

int oracle_adjoint_step(const oracle_cfg* c, const double* Sn, double dt, const double* alpha6, const double* lam_in,
                        double* lam_out) {
  if (check_cfg(c)) return -1;
  hwo::adjoint_step(*c, Sn, dt, alpha6, lam_in, lam_out);
  return 0;
}

// One HWENO stencil (Sec. 2.1) with all intermediates, for the unit tests.
// out[0..2] p_l(x_{i+1/2}); out[3] p0'(x_{i+1/2}); out[4..6] p_l'(x_i); out[7..9] beta_l; out[10] tau;
// out[11..13] omega^gamma; out[14..16] omega^d; out[17] u^-_{i+1/2}; out[18] v^-_{i+1/2};
// out[19] v~_i; out[20] u^+_{i-1/2}; out[21] v^+_{i-1/2}.
int oracle_stencil(const double* u3, const double* v2, double dx, double gamma0, double d0, double eps, int v_weighted,
                   double* out) {
  double g[3] = {gamma0, 0.5 * (1.0 - gamma0), 0.5 * (1.0 - gamma0)};
  double d[3] = {d0, 0.5 * (1.0 - d0), 0.5 * (1.0 - d0)};
  const bool vw = v_weighted != 0;
  hwo::StencilOut<double> o;
  hwo::hweno_stencil(u3[0], u3[1], u3[2], v2[0], v2[1], dx, g, d, eps, o, vw);
  for (int l = 0; l < 3; ++l) out[l] = o.p[l];
  out[3] = o.dp0;
  for (int l = 0; l < 3; ++l) out[4 + l] = o.dpc[l];
  for (int l = 0; l < 3; ++l) out[7 + l] = o.beta[l];
  out[10] = o.tau;
  for (int l = 0; l < 3; ++l) out[11 + l] = o.wg[l];
  for (int l = 0; l < 3; ++l) out[14 + l] = o.wd[l];
  out[17] = o.u_half;
  out[18] = o.v_half;
  out[19] = o.v_mod;
  hwo::interp_plus(u3[0], u3[1], u3[2], v2[0], v2[1], dx, g, eps, out[20], out[21], vw);
  return 0;
}

// D-terms of Eqs. (Cd-1), (DfDh): f4 = f_{i-1..i+2}, h2 = (h_{i-1}, h_{i+2}); out = (Df, Dh)
int oracle_dterms(const double* f4, const double* h2, double dx, double* out) {
  hwo::dterms(f4[0], f4[1], f4[2], f4[3], h2[0], h2[1], dx, out[0], out[1]);
  return 0;
}

// Eq. (Cd-2): h2 = (h_i, h_{i+1})
int oracle_dterms2(const double* f4, const double* h2, double dx, double* out) {
  hwo::dterms2(f4[0], f4[1], f4[2], f4[3], h2[0], h2[1], dx, out[0], out[1]);
  return 0;
}

// Euler pieces for the unit tests: flux, Jacobian, eigenvectors at a state.
int oracle_euler_flux(const oracle_cfg* c, int dir, const double* U, double* F) {
  if (check_cfg(c)) return -1;
  hwo::Phys<double>(*c).flux(dir, U, F);
  return 0;
}
int oracle_euler_jacobian(const oracle_cfg* c, int dir, const double* U, double* A) {
  if (check_cfg(c)) return -1;
  hwo::Phys<double>(*c).jacobian(dir, U, A);
  return 0;
}
// which = 0: Roe average of UL, UR; which = 1: the cell state UL.  R, L: m x m row major.
int oracle_euler_eigen(const oracle_cfg* c, int dir, int which, const double* UL, const double* UR, double* Rm,
                       double* Lm, double* state4) {
  if (check_cfg(c) || c->system != hwo::EULER) return -1;
  hwo::EigenState<double> s = which == 0 ? hwo::roe_average(*c, UL, UR) : hwo::cell_state(*c, UL);
  hwo::right_eigen(*c, dir, s, Rm);
  hwo::left_eigen(*c, dir, s, Lm);
  if (state4) {
    state4[0] = s.u;
    state4[1] = s.v;
    state4[2] = s.H;
    state4[3] = s.c;
  }
  return 0;
}

}  // extern "C"
