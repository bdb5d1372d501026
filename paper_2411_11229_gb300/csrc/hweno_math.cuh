// Device arithmetic of the HWENO-I scheme (Xie, Tao, Jiao, Zhang, arXiv 2411.11229), FP64.
//
// Everything here works in a direction-normalised frame: component 1 of a 2D Euler vector is the
// momentum normal to the face and component 2 the tangential one.  Callers permute components
// 1 <-> 2 when sweeping in y (the y Jacobian, flux and eigenvectors are the x ones with the two
// momenta and velocities exchanged).
//
// The forms below are algebraically identical to the paper's formulas but arranged for the
// FP64 pipe: one reciprocal per weight set (common denominator), shared smoothness indicators,
// factored eigenvector products, and derivatives carried as h*v to avoid divisions by h.
#pragma once
#include <cstdint>

namespace hw {

enum { SYS_ADV = 0, SYS_BURGERS = 1, SYS_EULER = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2 };

template <int DIM, int SYS>
struct Traits {
  static constexpr int NC = SYS == SYS_EULER ? (DIM == 1 ? 3 : 4) : 1;  // components
  static constexpr int NF = DIM + 1;                                    // fields U, V(, W)
  static constexpr int NG = DIM == 2 ? 3 : 2;  // nodal groups per direction: F, A*D_own(, A*D_other)
  static constexpr int NP = SYS == SYS_EULER ? (DIM == 2 ? 4 : 3) : 0;  // primitives per cell
};

// Parameters shared by all kernels of one grid.
struct Grid {
  int nx, ny;   // ny = 1 in 1D
  int bc;
  int pad_;
  long long plane;  // nx * ny
  double dx, dy, inv_dx, inv_dy;
  double gamma, gm1;
  double ax, ay;    // advection speeds
  double g0, g1;    // linear weights gamma0, gamma1 = gamma2 (Eq. interp)
  double d0, d1;    // limiter weights d0, d1 = d2 (Eq. limiter)
  double eps;       // epsilon of Eq. (nonlinear)
  double cfl;
};

__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
__device__ __forceinline__ double sqr(double x) { return x * x; }

// ---------------------------------------------------------------------------------------------
// Smoothness indicators (Eq. GHYZ, explicit forms) of the stencil {i-1, i, i+1} with values
// um, u0, up and scaled derivatives hvm = h v_{i-1}, hvp = h v_{i+1}.  beta0 is the paper's sum of
// four weighted squares, with a1..a4 regrouped as below.
struct Beta {
  double b0, b1, b2;
};

__device__ __forceinline__ Beta indicators(double um, double u0, double up, double hvm, double hvp) {
  const double sv = hvm + hvp, dv = hvm - hvp, du = up - um;
  const double d2 = fma(-2.0, u0, um + up);
  // a1 + a3/4 = -3/16 sv + 11/16 du;  a2 + 63/130 a4 = 67/520 dv + 197/260 d2;
  // a3 = (sv - du)/4;  a4 = -(dv/4 + d2/2)
  const double A = fma(-0.1875, sv, 0.6875 * du);
  const double B = fma(67.0 / 520.0, dv, (197.0 / 260.0) * d2);
  const double C = 0.25 * (sv - du);
  const double D = fma(0.25, dv, 0.5 * d2);
  Beta b;
  b.b0 = fma((1421461.0 / 2275.0) * D, D, fma((781.0 / 20.0) * C, C, fma((13.0 / 3.0) * B, B, A * A)));
  b.b1 = sqr(u0 - um);
  b.b2 = sqr(u0 - up);
  return b;
}

// Un-normalised nonlinear weights of Eq. (nonlinear) over the common denominator b0 b1 b2:
// omega_l is proportional to lin_l * W_l with W_l = (b_l + tau) * prod_{k != l} b_k, b = beta + eps.
struct Wts {
  double W0, W1, W2;
};

__device__ __forceinline__ Wts weights(const Beta& b, double eps) {
  const double tau_s = fabs(b.b0 - b.b1) + fabs(b.b0 - b.b2);
  const double tau = 0.25 * (tau_s * tau_s);
  const double e0 = b.b0 + eps, e1 = b.b1 + eps, e2 = b.b2 + eps;
  Wts w;
  w.W0 = (e0 + tau) * (e1 * e2);
  w.W1 = (e1 + tau) * (e0 * e2);
  w.W2 = (e2 + tau) * (e0 * e1);
  return w;
}

// u^-_{i+1/2} (Eqs. Pxi, interp) and h v^-_{i+1/2} = h p0'(x_{i+1/2}) (Eq. P'xi).
__device__ __forceinline__ void right_face(double um, double u0, double up, double hvm, double hvp, const Wts& w,
                                           double g0, double g1, double& u_out, double& hv_out) {
  const double p0 = fma(-0.125, um, fma(0.5625, u0 + up, fma(-0.046875, hvm, -0.140625 * hvp)));
  const double p1 = fma(-0.5, um, 1.5 * u0);
  const double p2 = 0.5 * (u0 + up);
  const double r = fma(-g1, p1 + p2, p0);
  const double num = fma(w.W0, r, g1 * fma(w.W1, p1, w.W2 * p2));
  const double den = fma(g0, w.W0, g1 * (w.W1 + w.W2));
  u_out = num * rcp(den);
  hv_out = fma(0.1875, um, fma(-1.5, u0, fma(1.3125, up, fma(0.0625, hvm, -0.1875 * hvp))));
}

// u^+_{i-1/2} and h v^+_{i-1/2}: the mirror image about x_i.  The linear candidate on {i, i+1}
// carries beta2 (W2) and the one on {i-1, i} carries beta1 (W1); gamma1 = gamma2.
__device__ __forceinline__ void left_face(double um, double u0, double up, double hvm, double hvp, const Wts& w,
                                          double g0, double g1, double& u_out, double& hv_out) {
  const double q0 = fma(0.5625, um + u0, fma(-0.125, up, fma(0.140625, hvm, 0.046875 * hvp)));
  const double q1 = fma(-0.5, up, 1.5 * u0);  // linear on {i, i+1}
  const double q2 = 0.5 * (um + u0);          // linear on {i-1, i}
  const double r = fma(-g1, q1 + q2, q0);
  const double num = fma(w.W0, r, g1 * fma(w.W2, q1, w.W1 * q2));
  const double den = fma(g0, w.W0, g1 * (w.W1 + w.W2));
  u_out = num * rcp(den);
  hv_out = fma(-1.3125, um, fma(1.5, u0, fma(-0.1875, up, fma(-0.1875, hvm, 0.0625 * hvp))));
}

// h v~_i (Eq. limiter with the derivatives of Eq. limiter-p) from the same W and the limiter's
// linear weights d0, d1 = d2.
__device__ __forceinline__ double limiter(double um, double u0, double up, double hvm, double hvp, const Wts& w,
                                          double d0, double d1) {
  const double du = up - um;
  const double hp0 = fma(0.75, du, -0.25 * (hvm + hvp));
  const double hp1 = u0 - um, hp2 = up - u0;
  const double num = fma(w.W0, fma(-d1, du, hp0), d1 * fma(w.W1, hp1, w.W2 * hp2));
  const double den = fma(d0, w.W0, d1 * (w.W1 + w.W2));
  return num * rcp(den);
}

// ---------------------------------------------------------------------------------------------
// Central Hermite correction (Eqs. Cd-1, DfDh) combined into its two stencils:
// D(f) = cf (f_{i-1} - f_i - f_{i+1} + f_{i+2}) + ch h (h_{i-1} - h_{i+2})
// D(h) = (1/h) (ef (f_{i-1} - f_{i+2}) + eg (f_{i+1} - f_i)) + eh (h_{i-1} + h_{i+2})
struct DCoef {
  static constexpr double cf = -(1.0 / 24.0) * (9.0 / 8.0) + (7.0 / 5760.0) * (-3.0);
  static constexpr double ch = -(1.0 / 24.0) * (5.0 / 12.0) + (7.0 / 5760.0) * (-2.0);
  static constexpr double ef = (1.0 / 24.0) * (101.0 / 36.0) + (7.0 / 5760.0) * (130.0 / 9.0);
  static constexpr double eg = (1.0 / 24.0) * (27.0 / 4.0) + (7.0 / 5760.0) * 30.0;
  static constexpr double eh = (1.0 / 24.0) * (5.0 / 6.0) + (7.0 / 5760.0) * (20.0 / 3.0);
};

// ---------------------------------------------------------------------------------------------
// Physics in the normal frame.  SPEED is the advection speed along the sweep direction.
template <int DIM, int SYS>
struct Phys;

template <int DIM>
struct Phys<DIM, SYS_ADV> {
  static constexpr int NC = 1;
  __device__ static void flux(const double* U, double* F, double a, double) { F[0] = a * U[0]; }
  __device__ static void jvp(const double*, const double* D, double* out, double a, double) { out[0] = a * D[0]; }
};

template <int DIM>
struct Phys<DIM, SYS_BURGERS> {
  static constexpr int NC = 1;
  __device__ static void flux(const double* U, double* F, double, double) { F[0] = 0.5 * (U[0] * U[0]); }
  __device__ static void jvp(const double* U, const double* D, double* out, double, double) { out[0] = U[0] * D[0]; }
};

// 1D Euler, U = (rho, m, E), p = (gamma-1)(E - m u / 2)
template <>
struct Phys<1, SYS_EULER> {
  static constexpr int NC = 3;
  __device__ static void flux(const double* U, double* F, double, double gm1) {
    const double ir = rcp(U[0]);
    const double u = U[1] * ir;
    const double p = gm1 * fma(-0.5 * U[1], u, U[2]);
    F[0] = U[1];
    F[1] = fma(U[1], u, p);
    F[2] = (U[2] + p) * u;
  }
  // A(U) D via the chain rule: u' = (m' - u rho')/rho, p' = (gamma-1)(E' - (m' u + m u')/2)
  __device__ static void jvp_prim(const double* U, double u, double p, double ir, const double* D, double* out,
                                  double gm1) {
    const double du = fma(-u, D[0], D[1]) * ir;
    const double dp = gm1 * fma(-0.5, fma(D[1], u, U[1] * du), D[2]);
    out[0] = D[1];
    out[1] = fma(D[1], u, fma(U[1], du, dp));
    out[2] = fma(D[2] + dp, u, (U[2] + p) * du);
  }
  __device__ static void jvp(const double* U, const double* D, double* out, double, double gm1) {
    const double ir = rcp(U[0]);
    const double u = U[1] * ir;
    const double p = gm1 * fma(-0.5 * U[1], u, U[2]);
    jvp_prim(U, u, p, ir, D, out, gm1);
  }
};

// 2D Euler in the normal frame, U = (rho, m_n, m_t, E)
template <>
struct Phys<2, SYS_EULER> {
  static constexpr int NC = 4;
  __device__ static void flux(const double* U, double* F, double, double gm1) {
    const double ir = rcp(U[0]);
    const double u = U[1] * ir, v = U[2] * ir;
    const double p = gm1 * fma(-0.5, fma(U[1], u, U[2] * v), U[3]);
    F[0] = U[1];
    F[1] = fma(U[1], u, p);
    F[2] = U[2] * u;
    F[3] = (U[3] + p) * u;
  }
  __device__ static void jvp_prim(const double* U, double u, double v, double p, double ir, const double* D,
                                  double* out, double gm1) {
    const double du = fma(-u, D[0], D[1]) * ir;
    const double dv = fma(-v, D[0], D[2]) * ir;
    // d/dx of (m u + n v)/2 = (m' u + m u' + n' v + n v')/2
    const double dk = fma(D[1], u, fma(U[1], du, fma(D[2], v, U[2] * dv)));
    const double dp = gm1 * fma(-0.5, dk, D[3]);
    out[0] = D[1];
    out[1] = fma(D[1], u, fma(U[1], du, dp));
    out[2] = fma(D[2], u, U[2] * du);
    out[3] = fma(D[3] + dp, u, (U[3] + p) * du);
  }
  __device__ static void jvp(const double* U, const double* D, double* out, double, double gm1) {
    const double ir = rcp(U[0]);
    const double u = U[1] * ir, v = U[2] * ir;
    const double p = gm1 * fma(-0.5, fma(U[1], u, U[2] * v), U[3]);
    jvp_prim(U, u, v, p, ir, D, out, gm1);
  }
};

// ---------------------------------------------------------------------------------------------
// Characteristic fields of the Euler equations in the normal frame.  Right eigenvectors
// (columns, ordered by eigenvalue): 1D (1, u-c, H-uc), (1, u, u^2/2), (1, u+c, H+uc);
// 2D (1, u-c, v, H-uc), (1, u, v, |q|^2/2), (0, 0, 1, v), (1, u+c, v, H+uc).
// Left eigenvectors applied in factored form with b1 = (gamma-1)/c^2, b2 = b1 |q|^2/2:
//   t = b2 q0 - b1 (u q1 + v q2 - q3), s = (u q0 - q1)/c,
//   w = ((t+s)/2, q0 - t, q2 - v q0, (t-s)/2)   [1D: no q2 term and no third row].
template <int NC>
struct Eig {
  double u, v, H, c;
  double hb1, hb2, hic;  // b1/2, b2/2, 1/(2c)
  double uc, hq2;        // u c, |q|^2 / 2

  __device__ void setup(double u_, double v_, double H_, double c_, double ic, double gm1) {
    u = u_;
    v = v_;
    H = H_;
    c = c_;
    const double q2 = NC == 4 ? fma(u, u, v * v) : u * u;
    hq2 = 0.5 * q2;
    hb1 = 0.5 * gm1 * (ic * ic);
    hb2 = hb1 * hq2;
    hic = 0.5 * ic;
    uc = u * c;
  }

  __device__ __forceinline__ void project(const double* q, double* w) const {
    double k = NC == 4 ? fma(v, q[2], u * q[1]) - q[3] : fma(u, q[1], -q[NC - 1]);
    const double th = fma(-hb1, k, hb2 * q[0]);  // t/2
    const double sh = fma(u, q[0], -q[1]) * hic;  // s/2
    w[0] = th + sh;
    w[1] = fma(-2.0, th, q[0]);
    if (NC == 4) {
      w[2] = fma(-v, q[0], q[2]);
      w[3] = th - sh;
    } else {
      w[2] = th - sh;
    }
  }

  __device__ __forceinline__ void back(const double* w, double* q) const {
    const double wl = w[0], wr = NC == 4 ? w[3] : w[2];
    const double sg = wl + wr, dl = wr - wl;
    q[0] = sg + w[1];
    q[1] = fma(u, q[0], c * dl);
    if (NC == 4) {
      q[2] = fma(v, q[0], w[2]);
      q[3] = fma(H, sg, fma(hq2, w[1], fma(v, w[2], uc * dl)));
    } else {
      q[2] = fma(H, sg, fma(hq2, w[1], uc * dl));
    }
  }
};

// ---------------------------------------------------------------------------------------------
// Boundary index maps.  Periodic wraps, transmissive clamps (zero-order extrapolation).
__device__ __forceinline__ int bc_index(int k, int n, int bc) {
  if (bc == BC_PERIODIC) {
    k = k < 0 ? k + n : k;
    return k >= n ? k - n : k;
  }
  return k < 0 ? 0 : (k >= n ? n - 1 : k);
}

__device__ __forceinline__ unsigned long long dbl_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

}  // namespace hw
