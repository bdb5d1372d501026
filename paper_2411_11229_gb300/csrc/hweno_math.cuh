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
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_FIXED = 3 };
// scheme variants of the extended kernels (VAR != 0)
enum { FLAG_V_WEIGHTED = 1, FLAG_CD2 = 2, FLAG_R2 = 4, FLAG_ALPHA_STEP = 8, FLAG_ALPHA_LOCAL = 16 };

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
  int flags;    // FLAG_* (read by the extended kernels only)
  long long plane;  // nx * ny
  double dx, dy, inv_dx, inv_dy;
  double gamma, gm1;
  double ax, ay;    // advection speeds
  double g0, g1;    // linear weights gamma0, gamma1 = gamma2 (Eq. interp)
  double d0, d1;    // limiter weights d0, d1 = d2 (Eq. limiter)
  double eps;       // epsilon of Eq. (nonlinear)
  double cfl;
  // Folded constants (computed on the host from the linear weights and the spacings):
  //   cr, cl: coefficients of (p0 - gamma1 (p1 + p2)) / gamma1 on (um, u0, up, hvm, hvp) at the
  //           right face x_{i+1/2} and, mirrored, at the left face x_{i-1/2};
  //   G = gamma0 / gamma1;  limiter: cdu = (3/4 - d1)/d1, Gd = d0 / d1;
  //   per direction: h, 1/h, ch*h, ef/h, eg/h (D-terms), 1/(2h).
  double cr[5], cl[5], G;
  double cdu, Gd;
  // The arithmetic with the derivatives entering unscaled (v, not h v), per direction: the h of
  // every derivative term folded into its coefficient (the forward and the adjoint kernels).
  // bS1, bN1, bS2, bN2 (per direction) and bT1, bT2: the smoothness indicator as
  // S1 (sv + N1 du)^2 + T1 du^2 + S2 (dv + N2 d2)^2 + T2 d2^2 (see beta0_eps); udm, udp: the
  // combinations (p0 - gamma1 (p1 + p2))/gamma1 - G u_i with the centre value taken out (their value
  // coefficients sum to G) on (d01, d12, vm, vp) at the right face and, mirrored, on
  // (d_{i-1,i}, d_{i,i+1}, ...) at the left face; uvd = (21/16, 3/16)/h: the cell differences in
  // the derivative at the face; ucsv = h/(4 d1), the limiter's derivative coefficient.
  double bS1[2], bN1[2], bS2[2], bN2[2], bT1, bT2;
  double udm[2][4], udp[2][4], uvd[2][2], ucsv[2];
  double h[2], ih[2], chh[2], efih[2], egih[2], hih[2];
  // Extended scheme (read only by the kernels instantiated with VAR != 0):
  //   side: boundary type of x-low, x-high, y-low, y-high; grav: g of Eq. (euler2d-s);
  //   ig1 = 1/gamma1 (weighted derivative); Cd-2 folded per direction: c2h = c2 h,
  //   e2fih = e2f/h, e2gih = e2g/h;
  //   fixU, fixP, fixF: the state of a BC_FIXED side (original frame), its primitives
  //   (sqrt rho, u[, v], H) and its flux normal to the side (normal frame); fixA: its spectral
  //   radius normal to the side (local LF coefficient).
  int side[4];
  double grav, ig1;
  double c2h[2], e2fih[2], e2gih[2];
  double fixU[4][4], fixP[4][4], fixF[4][4], fixA[4];
};

// FP64 issue on this GPU (measured with independent chains per thread): a DFMA whose three operands
// are thread registers issues at 1.9 per SM-clock; DADD, DMUL, and a DFMA with an immediate,
// constant-bank or block-uniform operand, at 1.6.  The stage and adjoint kernels therefore issue
// their sums, differences and products of register values as DFMAs against 1 and -0 held in thread
// registers:
// fma(a, 1, b) = a + b and fma(a, b, -0) = a b exactly (the same rounding, signed zeros included).
// FU carries the two units; the kernels load them through memory the compiler cannot see into
// (fu_of), and the default FU{1, -0, 0} folds back to plain sums and products.  reg(c) copies a
// constant into a thread register through the integer pipe (its bits XOR a zero the compiler cannot
// see), so that the DFMAs reading it take register operands at no FP64 issue slot.
struct FU {
  double one, mz;
  int zi;  // 0
  __device__ __forceinline__ double add(double a, double b) const { return fma(a, one, b); }
  __device__ __forceinline__ double sub(double a, double b) const { return fma(a, one, -b); }
  __device__ __forceinline__ double mul(double a, double b) const { return fma(a, b, mz); }
  __device__ __forceinline__ double reg(double c) const {
    return __hiloint2double(__double2hiint(c) ^ zi, __double2loint(c) ^ zi);
  }
};
#define HW_PLAIN_FU FU{1.0, -0.0, 0}

// 1/x for normal, finite x: the hardware approximation (rcp.approx.ftz.f64, relative error up to
// about 2^-20 on this GPU) refined by one third-order step.  With e = 1 - x r the exact reciprocal
// is r / (1 - e) = r (1 + e + e^2 + ...); keeping the series to e^2 leaves a relative error of
// order e^3 (about 2^-60), so the result is within one unit in the last place (measured: 1 ulp at
// most, on 0.03 % of inputs).  Three FMAs, against four for two Newton-Raphson steps
// r <- r + r (1 - x r).
__device__ __forceinline__ double rcp(double x, const FU& f = HW_PLAIN_FU) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, f.one);
  return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double sqr(double x) { return x * x; }

// ---------------------------------------------------------------------------------------------
// Smoothness indicators (Eq. GHYZ, explicit forms) of the stencil {i-1, i, i+1} from the cell
// differences dm = u_i - u_{i-1}, dp = u_{i+1} - u_i and the scaled derivatives hvm = h v_{i-1},
// hvp = h v_{i+1}:  with du = dm + dp, d2 = dp - dm, sv = hvm + hvp, dv = hvm - hvp,
//   a1 + a3/4 = -3/16 sv + 11/16 du,  a2 + 63/130 a4 = 67/520 dv + 197/260 d2,
//   a3 = (sv - du)/4,  a4 = -(dv + 2 d2)/4,
// beta0 = (a1 + a3/4)^2 + 13/3 (a2 + 63/130 a4)^2 + 781/20 a3^2 + 1421461/2275 a4^2,
// beta1 = dm^2, beta2 = dp^2 (passed in: neighbouring stencils share them).  The kernels evaluate
// beta0 through the completed squares below (beta0_eps; the adjoint's beta0_eps_s).

// The constants of one direction's stencils (Grid fields of that direction, see Grid), copied into
// thread registers by stencil_k: a DFMA issues faster with register operands than with a
// constant-bank or block-uniform one (see FU), and every stencil of a face or cell reads them.
struct StencilK {
  double bN1, bN2, bS1, bS2, bT1, bT2, eps;  // beta0 + eps (beta0_eps)
  double quarter, half;                      // 1/4 of tau, 1/2 of the candidate slopes
  double G, cm[4], cp[4];                    // face: gamma0/gamma1, udm and udp of the direction
  double cdu, mucsv, Gd, ih;                 // cell: the limiter's cdu, -ucsv, d0/d1 and 1/h
};
// k = the stencil constants of direction dir, copied into thread registers (FU::reg; with the
// default units the compiler keeps them as the constants)
__device__ __forceinline__ StencilK stencil_k(const Grid& g, int dir, const FU& f = HW_PLAIN_FU) {
  StencilK k;
  k.bN1 = f.reg(g.bN1[dir]);
  k.bN2 = f.reg(g.bN2[dir]);
  k.bS1 = f.reg(g.bS1[dir]);
  k.bS2 = f.reg(g.bS2[dir]);
  k.bT1 = f.reg(g.bT1);
  k.bT2 = f.reg(g.bT2);
  k.eps = f.reg(g.eps);
  k.quarter = f.reg(0.25);
  k.half = f.reg(0.5);
  k.G = f.reg(g.G);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    k.cm[i] = f.reg(g.udm[dir][i]);
    k.cp[i] = f.reg(g.udp[dir][i]);
  }
  k.cdu = f.reg(g.cdu);
  k.mucsv = f.reg(-g.ucsv[dir]);
  k.Gd = f.reg(g.Gd);
  k.ih = f.reg(g.ih[dir]);
  return k;
}

// beta0 + eps with unscaled derivatives vm = v_{i-1}, vp = v_{i+1} along the direction of k.  The
// four squared forms of beta0 make one quadratic form in (h sv, du) and one in (h dv, d2);
// completing the square in the derivative term writes them as S1 (sv + N1 du)^2 + T1 du^2 and
// S2 (dv + N2 d2)^2 + T2 d2^2 (S, N per direction, T independent of h), a sum of four non-negative
// terms, and eps enters as the first addend.  Returns beta0 + eps, du = dm + dp and sv = vm + vp.
__device__ __forceinline__ double beta0_eps(double dm, double dp, double vm, double vp, const StencilK& k,
                                            double& du_out, double& sv_out, const FU& f = HW_PLAIN_FU) {
  const double du = f.add(dm, dp), d2 = f.sub(dp, dm);
  const double sv = f.add(vm, vp), dv = f.sub(vm, vp);
  const double y1 = fma(k.bN1, du, sv), y2 = fma(k.bN2, d2, dv);
  du_out = du;
  sv_out = sv;
  return fma(f.mul(k.bS1, y1), y1,
             fma(f.mul(k.bS2, y2), y2, fma(f.mul(k.bT1, du), du, fma(f.mul(k.bT2, d2), d2, k.eps))));
}

// Nonlinear weights of Eq. (nonlinear) up to a common factor: with e_l = beta_l + eps,
// omega_l is proportional to lin_l (1 + tau/e_l), i.e. to lin_l W_l with
// W_l = e0 e1 e2 + tau * prod_{k != l} e_k.  One reciprocal normalises them later.
struct Wts {
  double W0, W1, W2;
  double tau;  // tau of Eq. (nonlinear) (read by the adjoint's saved forward pass)
};

// Weights from e_l = beta_l + eps directly: e_l - e_k stands for beta_l - beta_k in tau.  quarter:
// 1/4 (a register copy where the caller has one).
__device__ __forceinline__ Wts weights_e(double e0, double e1, double e2, double quarter, const FU& f = HW_PLAIN_FU) {
  const double ts = f.add(fabs(f.sub(e0, e1)), fabs(f.sub(e0, e2)));
  const double tau = f.mul(f.mul(quarter, ts), ts);
  const double Q0 = f.mul(e1, e2), Q1 = f.mul(e0, e2), Q2 = f.mul(e0, e1);
  const double P = f.mul(Q0, e0);
  Wts w;
  w.W0 = fma(tau, Q0, P);
  w.W1 = fma(tau, Q1, P);
  w.W2 = fma(tau, Q2, P);
  w.tau = tau;
  return w;
}
__device__ __forceinline__ Wts weights_e(double e0, double e1, double e2, const FU& f = HW_PLAIN_FU) {
  return weights_e(e0, e1, e2, 0.25, f);
}

// One characteristic field at one face k+1/2: u^- from the stencil of cell k (Eqs. Pxi, P'xi,
// interp) and u^+ from the stencil of cell k+1 evaluated at its left face (the mirror image about
// x_{k+1}); gamma1 = gamma2, and each weight set normalises with one reciprocal.  Every candidate
// reproduces constants and the candidates' value coefficients sum to G, so each value is the centre
// value plus a combination of cell differences:
//   num / den = u_c + (W0 (r - G u_c) + W1 (p1 - u_c) + W2 (p2 - u_c)) / den,
// with p1 - u_c and p2 - u_c half a cell difference each.  In: d01 = w1 - w0, d12 = w2 - w1,
// d23 = w3 - w2 over the cells k-1..k+2 and their derivatives y0..y3 along direction dir
// (unscaled); k: the stencil constants of dir.  Out: um, up = the interface values less the centre
// values w1, w2, added to bm, bp (the centre values for a scalar law, zero where the caller adds the
// centre states in conserved variables); with VW (the weighted-derivative option), the weighted
// derivatives vm, vp (the unweighted ones are linear in the stencil and formed by the caller).
template <bool VW>
__device__ __forceinline__ void face_field_d(double d01, double d12, double d23, double y0, double y1, double y2,
                                             double y3, double bm, double bp, const StencilK& k, const Grid& g,
                                             int dir, double& um, double& vm, double& up, double& vp,
                                             const FU& f = HW_PLAIN_FU) {
  const double e01 = fma(d01, d01, k.eps), e12 = fma(d12, d12, k.eps), e23 = fma(d23, d23, k.eps);
  const double k21 = g.uvd[dir][0], k3 = g.uvd[dir][1];
  vm = vp = 0.0;
  double du, sv;
  {
    // stencil of cell k: candidates on {i-1, i} (W1), {i, i+1} (W2)
    const double e0 = beta0_eps(d01, d12, y0, y2, k, du, sv, f);
    const Wts wt = weights_e(e0, e01, e12, k.quarter, f);
    const double r = fma(k.cm[0], d01, fma(k.cm[1], d12, fma(k.cm[2], y0, f.mul(k.cm[3], y2))));
    const double sl = fma(wt.W1, d01, f.mul(wt.W2, d12));
    const double rden = rcp(fma(k.G, wt.W0, f.add(wt.W1, wt.W2)), f);
    um = fma(fma(wt.W0, r, f.mul(k.half, sl)), rden, bm);
    if (VW) {
      const double ih = g.ih[dir];
      const double v0 = fma(k21, d12, fma(-k3, d01, fma(0.0625, y0, -0.1875 * y2)));
      vm = f.mul(fma(wt.W0, fma(v0, g.ig1, -du * ih), sl * ih), rden);
    }
  }
  {
    // stencil of cell k+1 (mirror image): its candidate on {i, i+1} carries beta2
    const double e0 = beta0_eps(d12, d23, y1, y3, k, du, sv, f);
    const Wts wt = weights_e(e0, e12, e23, k.quarter, f);
    const double r = fma(k.cp[0], d12, fma(k.cp[1], d23, fma(k.cp[2], y1, f.mul(k.cp[3], y3))));
    const double sl = fma(wt.W1, d12, f.mul(wt.W2, d23));
    const double rden = rcp(fma(k.G, wt.W0, f.add(wt.W1, wt.W2)), f);
    up = fma(fma(wt.W0, r, -f.mul(k.half, sl)), rden, bp);
    if (VW) {
      const double ih = g.ih[dir];
      const double v0 = fma(k21, d12, fma(-k3, d23, fma(-0.1875, y1, 0.0625 * y3)));
      vp = f.mul(fma(wt.W0, fma(v0, g.ig1, -du * ih), sl * ih), rden);
    }
  }
}

// R2 variant: one characteristic field of cell i from its own stencil, on differences
// d01 = w1 - w0, d12 = w2 - w1 and unscaled derivatives y0 = v_{i-1}, y2 = v_{i+1}: u^- at
// x_{i+1/2} and u^+ at x_{i-1/2} less the centre value, added to bc (as in face_field_d), with VW
// the weighted derivatives v^- and v^+, and h v~_i.  The three share beta, tau and the unnormalised
// weights; u^+/- share one reciprocal (gamma1 = gamma2 makes the mirrored weights the same numbers).
template <bool VW>
__device__ __forceinline__ void cell_faces_field(double d01, double d12, double y0, double y2, double bc,
                                                 const StencilK& k, const Grid& g, int dir, double& um, double& vm,
                                                 double& up, double& vp, double& hvt, const FU& f = HW_PLAIN_FU) {
  double du, sv;
  const double e0 = beta0_eps(d01, d12, y0, y2, k, du, sv, f);
  const Wts wt = weights_e(e0, fma(d01, d01, k.eps), fma(d12, d12, k.eps), k.quarter, f);
  const double rden = rcp(fma(k.G, wt.W0, f.add(wt.W1, wt.W2)), f);
  // the candidates at x_{i+1/2} differ from u_i by (d01, d12)/2, those at x_{i-1/2} by
  // (-d01, -d12)/2, so both faces share W1 d01 + W2 d12
  const double rm = fma(k.cm[0], d01, fma(k.cm[1], d12, fma(k.cm[2], y0, f.mul(k.cm[3], y2))));
  const double rp = fma(k.cp[0], d01, fma(k.cp[1], d12, fma(k.cp[2], y0, f.mul(k.cp[3], y2))));
  const double sl = fma(wt.W1, d01, f.mul(wt.W2, d12));
  const double hs = f.mul(k.half, sl);
  um = fma(fma(wt.W0, rm, hs), rden, bc);
  up = fma(fma(wt.W0, rp, -hs), rden, bc);
  vm = vp = 0.0;
  if (VW) {
    const double k21 = g.uvd[dir][0], k3 = g.uvd[dir][1];
    const double ih = g.ih[dir], ds = du * ih, ss = sl * ih;
    const double v0m = fma(k21, d12, fma(-k3, d01, fma(0.0625, y0, -0.1875 * y2)));
    const double v0p = fma(k21, d01, fma(-k3, d12, fma(-0.1875, y0, 0.0625 * y2)));
    vm = f.mul(fma(wt.W0, fma(v0m, g.ig1, -ds), ss), rden);
    vp = f.mul(fma(wt.W0, fma(v0p, g.ig1, -ds), ss), rden);
  }
  const double t = fma(k.cdu, du, f.mul(k.mucsv, sv));
  hvt = f.mul(fma(wt.W0, t, sl), rcp(fma(k.Gd, wt.W0, f.add(wt.W1, wt.W2)), f));
}

// h v~_i of one characteristic field (Eq. limiter with the derivatives of Eq. limiter-p) from the
// differences d01 = w1 - w0, d12 = w2 - w1 of u_{i-1..i+1} and the unscaled derivatives
// y0 = v_{i-1}, y2 = v_{i+1} along the direction of k:
//   (h p0'(x_i) - d1 (h p1' + h p2')) / d1 = cdu du - csv h sv,  h p1' = d01, h p2' = d12.
__device__ __forceinline__ double cell_field_d(double d01, double d12, double y0, double y2, const StencilK& k,
                                               const FU& f = HW_PLAIN_FU) {
  double du, sv;
  const double e0 = beta0_eps(d01, d12, y0, y2, k, du, sv, f);
  const Wts wt = weights_e(e0, fma(d01, d01, k.eps), fma(d12, d12, k.eps), k.quarter, f);
  const double t = fma(k.cdu, du, f.mul(k.mucsv, sv));
  const double num = fma(wt.W0, t, fma(wt.W1, d01, f.mul(wt.W2, d12)));
  const double den = fma(k.Gd, wt.W0, f.add(wt.W1, wt.W2));
  return f.mul(num, rcp(den, f));
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

// The alternative D-terms of Eq. (Cd-2) (h at the two inner nodes), combined the same way:
// D(f) = c2f (f_{i-1} - f_i - f_{i+1} + f_{i+2}) + c2 h (h_i - h_{i+1})
// D(h) = (1/h) (e2f (f_{i-1} - f_{i+2}) + e2g (f_i - f_{i+1})) + e2h (h_i + h_{i+1})
struct DCoef2 {
  static constexpr double cf = -(1.0 / 24.0) * (-1.0 / 8.0) + (7.0 / 5760.0) * 3.0;
  static constexpr double ch = -(1.0 / 24.0) * (-5.0 / 4.0) + (7.0 / 5760.0) * 6.0;
  static constexpr double ef = -(1.0 / 24.0) * (1.0 / 4.0) + (7.0 / 5760.0) * (-10.0);
  static constexpr double eg = -(1.0 / 24.0) * (57.0 / 4.0) + (7.0 / 5760.0) * (-90.0);
  static constexpr double eh = -(1.0 / 24.0) * (15.0 / 2.0) + (7.0 / 5760.0) * (-60.0);
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
  __device__ static void flux_jvp(const double* U, const double* D, double* F, double* out, double a, double gm1,
                                  const FU& = HW_PLAIN_FU) {
    flux(U, F, a, gm1);
    jvp(U, D, out, a, gm1);
  }
};

template <int DIM>
struct Phys<DIM, SYS_BURGERS> {
  static constexpr int NC = 1;
  __device__ static void flux(const double* U, double* F, double, double) { F[0] = 0.5 * (U[0] * U[0]); }
  __device__ static void jvp(const double* U, const double* D, double* out, double, double) { out[0] = U[0] * D[0]; }
  __device__ static void flux_jvp(const double* U, const double* D, double* F, double* out, double a, double gm1,
                                  const FU& = HW_PLAIN_FU) {
    flux(U, F, a, gm1);
    jvp(U, D, out, a, gm1);
  }
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
                                  double gm1, const FU& f = HW_PLAIN_FU) {
    const double du = f.mul(fma(-u, D[0], D[1]), ir);
    const double dp = gm1 * fma(-0.5, fma(D[1], u, f.mul(U[1], du)), D[2]);
    out[0] = D[1];
    out[1] = fma(D[1], u, fma(U[1], du, dp));
    out[2] = fma(f.add(D[2], dp), u, f.mul(f.add(U[2], p), du));
  }
  __device__ static void jvp(const double* U, const double* D, double* out, double, double gm1) {
    const double ir = rcp(U[0]);
    const double u = U[1] * ir;
    const double p = gm1 * fma(-0.5 * U[1], u, U[2]);
    jvp_prim(U, u, p, ir, D, out, gm1);
  }
  // f(U) and A(U) D with one reciprocal and one pressure
  __device__ static void flux_jvp(const double* U, const double* D, double* F, double* out, double, double gm1,
                                  const FU& f = HW_PLAIN_FU) {
    const double ir = rcp(U[0], f);
    const double u = f.mul(U[1], ir);
    const double p = gm1 * fma(-0.5 * U[1], u, U[2]);
    F[0] = U[1];
    F[1] = fma(U[1], u, p);
    F[2] = f.mul(f.add(U[2], p), u);
    jvp_prim(U, u, p, ir, D, out, gm1, f);
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
                                  double* out, double gm1, const FU& f = HW_PLAIN_FU) {
    const double du = f.mul(fma(-u, D[0], D[1]), ir);
    const double dv = f.mul(fma(-v, D[0], D[2]), ir);
    // d/dx of (m u + n v)/2 = (m' u + m u' + n' v + n v')/2
    const double dk = fma(D[1], u, fma(U[1], du, fma(D[2], v, f.mul(U[2], dv))));
    const double dp = gm1 * fma(-0.5, dk, D[3]);
    out[0] = D[1];
    out[1] = fma(D[1], u, fma(U[1], du, dp));
    out[2] = fma(D[2], u, f.mul(U[2], du));
    out[3] = fma(f.add(D[3], dp), u, f.mul(f.add(U[3], p), du));
  }
  __device__ static void jvp(const double* U, const double* D, double* out, double, double gm1) {
    const double ir = rcp(U[0]);
    const double u = U[1] * ir, v = U[2] * ir;
    const double p = gm1 * fma(-0.5, fma(U[1], u, U[2] * v), U[3]);
    jvp_prim(U, u, v, p, ir, D, out, gm1);
  }
  // The derivatives of the primitives along D (original frame): u' = (m' - u rho')/rho,
  // v' = (n' - v rho')/rho, p' = (gamma-1)(E' - (m' u + m u' + n' v + n v')/2).  They do not depend
  // on the direction, so a cell computes them once per derivative field for both Jacobians.
  __device__ static void prim_deriv(const double* U, double u, double v, double ir, const double* D, double gm1,
                                    double& du, double& dv, double& dp, const FU& f = HW_PLAIN_FU) {
    du = f.mul(fma(-u, D[0], D[1]), ir);
    dv = f.mul(fma(-v, D[0], D[2]), ir);
    const double dk = fma(D[1], u, fma(U[1], du, fma(D[2], v, f.mul(U[2], dv))));
    dp = gm1 * fma(-0.5, dk, D[3]);
  }
  // A(U) D in the normal frame from the primitive derivatives: Un, Dn normal-frame vectors, un
  // the normal velocity, dun its derivative, hp = E + p
  __device__ static void jvp_apply(const double* Un, const double* Dn, double un, double dun, double dp, double hp,
                                   double* out, const FU& f = HW_PLAIN_FU) {
    out[0] = Dn[1];
    out[1] = fma(Dn[1], un, fma(Un[1], dun, dp));
    out[2] = fma(Dn[2], un, f.mul(Un[2], dun));
    out[3] = fma(f.add(Dn[3], dp), un, f.mul(hp, dun));
  }
  // f(U) and A(U) D with one reciprocal and one pressure
  __device__ static void flux_jvp(const double* U, const double* D, double* F, double* out, double, double gm1,
                                  const FU& f = HW_PLAIN_FU) {
    const double ir = rcp(U[0], f);
    const double u = f.mul(U[1], ir), v = f.mul(U[2], ir);
    const double p = gm1 * fma(-0.5, fma(U[1], u, f.mul(U[2], v)), U[3]);
    F[0] = U[1];
    F[1] = fma(U[1], u, p);
    F[2] = f.mul(U[2], u);
    F[3] = f.mul(f.add(U[3], p), u);
    jvp_prim(U, u, v, p, ir, D, out, gm1, f);
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

  __device__ __forceinline__ void project(const double* q, double* w, const FU& f = HW_PLAIN_FU) const {
    double k = NC == 4 ? f.sub(fma(v, q[2], f.mul(u, q[1])), q[3]) : fma(u, q[1], -q[NC - 1]);
    const double th = fma(-hb1, k, f.mul(hb2, q[0]));  // t/2
    const double sh = f.mul(fma(u, q[0], -q[1]), hic);  // s/2
    w[0] = f.add(th, sh);
    w[1] = fma(-2.0, th, q[0]);
    if (NC == 4) {
      w[2] = fma(-v, q[0], q[2]);
      w[3] = f.sub(th, sh);
    } else {
      w[2] = f.sub(th, sh);
    }
  }

  // q = base + R w: the interface state as the centre state plus the back-projected correction
  __device__ __forceinline__ void back_add(const double* w, const double* base, double* q,
                                           const FU& f = HW_PLAIN_FU) const {
    const double wl = w[0], wr = NC == 4 ? w[3] : w[2];
    const double sg = f.add(wl, wr), dl = f.sub(wr, wl);
    const double q0 = f.add(sg, w[1]);
    q[0] = f.add(base[0], q0);
    q[1] = fma(u, q0, fma(c, dl, base[1]));
    if (NC == 4) {
      q[2] = fma(v, q0, f.add(w[2], base[2]));
      q[3] = fma(H, sg, fma(hq2, w[1], fma(v, w[2], fma(uc, dl, base[3]))));
    } else {
      q[2] = fma(H, sg, fma(hq2, w[1], fma(uc, dl, base[2])));
    }
  }

  __device__ __forceinline__ void back(const double* w, double* q, const FU& f = HW_PLAIN_FU) const {
    const double wl = w[0], wr = NC == 4 ? w[3] : w[2];
    const double sg = f.add(wl, wr), dl = f.sub(wr, wl);
    q[0] = f.add(sg, w[1]);
    q[1] = fma(u, q[0], f.mul(c, dl));
    if (NC == 4) {
      q[2] = fma(v, q[0], w[2]);
      q[3] = fma(H, sg, fma(hq2, w[1], fma(v, w[2], f.mul(uc, dl))));
    } else {
      q[2] = fma(H, sg, fma(hq2, w[1], f.mul(uc, dl)));
    }
  }
};

// ---------------------------------------------------------------------------------------------
// Bounds-checked build (-DHWENO_BOUNDS_CHECK: libhweno_bounds.so, a debugging aid in place of a
// memory checker).  Every array access of the kernels is base + (field NC + comp) extent + index,
// with field and comp bounded by compile-time constants and each base and extent fixed by the host
// layout, so checking each cell, face and ghost-line index where a kernel forms it covers the
// accesses.  HW_IDX(i, n) is i when 0 <= i < n; otherwise it counts the event, records the source
// line of the first one, and gives 0, so that the access stays inside its array.  The host reads
// and clears the record with bounds_take (one record per translation unit; hweno_bounds_status).
// In the normal build HW_IDX(i, n) is i.
#ifdef HWENO_BOUNDS_CHECK
static __device__ unsigned int g_bounds_count;
static __device__ int g_bounds_line;
__device__ __forceinline__ long long bounds_idx(long long i, long long n, int line) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&g_bounds_count, 1u) == 0u) g_bounds_line = line;
  return 0;
}
#define HW_IDX(i, n) ::hw::bounds_idx((long long)(i), (long long)(n), __LINE__)
// this translation unit's count of out-of-range indices since the last call, and the source line
// of the first (synchronous copies; clears the count)
[[maybe_unused]] static unsigned int bounds_take(int* line) {
  unsigned int c = 0, z = 0;
  int l = 0;
  cudaMemcpyFromSymbol(&c, g_bounds_count, sizeof c);
  cudaMemcpyFromSymbol(&l, g_bounds_line, sizeof l);
  cudaMemcpyToSymbol(g_bounds_count, &z, sizeof z);
  if (line) *line = l;
  return c;
}
#else
#define HW_IDX(i, n) (i)
#endif

// ---------------------------------------------------------------------------------------------
// Boundary index maps.  Periodic wraps, transmissive clamps (zero-order extrapolation),
// reflective mirrors about the wall (cell -1-k for k < 0, 2n-1-k for k >= n) and sets refl.
__device__ __forceinline__ int bc_map(int k, int n, int bc, bool& refl) {
  refl = false;
  if (k >= 0 && k < n) return k;
  if (bc == BC_PERIODIC) return k < 0 ? k + n : k - n;
  if (bc == BC_TRANSMISSIVE) return k < 0 ? 0 : n - 1;
  refl = true;
  return k < 0 ? -1 - k : 2 * n - 1 - k;
}

// Per-side version for the extended kernels: lo and hi are the types of the two ends of the
// axis.  A BC_FIXED ghost sets fixed and returns the nearest interior index (its loads are then
// replaced by the side's state, so every load stays in bounds).
__device__ __forceinline__ int bc_map_ext(int k, int n, int lo, int hi, bool& refl, bool& fixed) {
  refl = false;
  fixed = false;
  if (k >= 0 && k < n) return k;
  const int t = k < 0 ? lo : hi;
  if (t == BC_FIXED) {
    fixed = true;
    return k < 0 ? 0 : n - 1;
  }
  return bc_map(k, n, t, refl);
}

__device__ __forceinline__ int bc_index(int k, int n, int bc) {
  bool refl;
  return bc_map(k, n, bc, refl);
}

// -x when b, else x: a flip of the sign bit in the integer pipe, so that a data-dependent sign
// costs no FP64 instruction
__device__ __forceinline__ double neg_if(double x, bool b) {
  return __hiloint2double(__double2hiint(x) ^ (b ? (int)0x80000000 : 0), __double2loint(x));
}

// A mirrored cell in the normal frame (Eqs. RBC-1d, RBC-2d-x, RBC-2d-y):
// in U and in the tangential derivative the normal momentum changes sign; in the normal derivative
// every component except that of the normal momentum changes sign.  Its nodal values then follow
// exactly: f -> -sU f, f'(u) v (normal derivative) -> sU (f'(u) v), mixed value -> -sU (...),
// with sU = -1 for the normal momentum and +1 otherwise.
template <int NC>
__device__ __forceinline__ void mirror_U(double* q, bool b) {
  q[1] = neg_if(q[1], b);
}
template <int NC>
__device__ __forceinline__ void mirror_D(double* q, bool b) {
#pragma unroll
  for (int k = 0; k < NC; ++k)
    if (k != 1) q[k] = neg_if(q[k], b);
}

__device__ __forceinline__ unsigned long long dbl_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

}  // namespace hw
