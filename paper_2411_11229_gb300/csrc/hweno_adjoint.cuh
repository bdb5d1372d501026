// Reverse-mode derivatives (hand-written) of the device arithmetic in hweno_math.cuh, for the
// adjoint of one Runge-Kutta stage.  Conventions: the LF coefficient alpha of every stage and the
// step size are held fixed; d|x|/dx = sign(x) with sign(0) = 0 (mul_sgn).  Every backward routine
// reads the forward values it needs (saved by the forward pass or recomputed from the same inputs)
// and ADDS the adjoints of its inputs to the bar arrays.
#pragma once
#include "hweno_kernels.cuh"

namespace hw {

// The stencil constants of one direction, those of the forward kernels (StencilK): derivatives
// enter unscaled, the h of every derivative term folded into its coefficient (see Grid).  Copied
// into thread registers through the integer pipe (FU::reg) so that the DFMAs reading them take
// register operands: the indicator's split (aN = bN[dir], aS = bS[dir], bT), eps, G, Gd, cdu,
// csv = ucsv[dir] and the candidate coefficients dm = udm[dir], dp = udp[dir].
struct AdjK {
  double eps, aN1, aN2, aS1, aS2, bT1, bT2, G, Gd, cdu, csv;
  double dm[4], dp[4];
};
__device__ __forceinline__ AdjK adj_k(const Grid& g, int dir, const FU& f) {
  AdjK k;
  k.eps = f.reg(g.eps);
  k.aN1 = f.reg(g.bN1[dir]);
  k.aN2 = f.reg(g.bN2[dir]);
  k.aS1 = f.reg(g.bS1[dir]);
  k.aS2 = f.reg(g.bS2[dir]);
  k.bT1 = f.reg(g.bT1);
  k.bT2 = f.reg(g.bT2);
  k.G = f.reg(g.G);
  k.Gd = f.reg(g.Gd);
  k.cdu = f.reg(g.cdu);
  k.csv = f.reg(g.ucsv[dir]);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    k.dm[i] = f.reg(g.udm[dir][i]);
    k.dp[i] = f.reg(g.udp[dir][i]);
  }
  return k;
}

// e0 = beta0 + eps of the stencil {i-1, i, i+1} from the differences dm, dp and the unscaled
// derivatives ym = v_{i-1}, yp = v_{i+1} along the direction of k (Eq. GHYZ; the forward kernels'
// beta0_eps): the two quadratic forms of beta0 with the square completed in the derivative term, S1 (sv + N1 du)^2 + T1 du^2 + S2 (dv + N2 d2)^2 + T2 d2^2
// (du = dm + dp, d2 = dp - dm, sv = ym + yp, dv = ym - yp), eps as the first addend.  Returns e0,
// du and sv, and in bt the four products S1 y1, S2 y2, T1 du, T2 d2 (its backward pass reads them).
struct BetaTerms {
  double s1y1, s2y2, t1du, t2d2;
};
__device__ __forceinline__ double beta0_eps_s(double dm, double dp, double ym, double yp, const AdjK& k, const FU& f,
                                              double& du_out, double& sv_out, BetaTerms& bt) {
  const double du = f.add(dm, dp), d2 = f.sub(dp, dm);
  const double sv = f.add(ym, yp), dv = f.sub(ym, yp);
  const double y1 = fma(k.aN1, du, sv), y2 = fma(k.aN2, d2, dv);
  du_out = du;
  sv_out = sv;
  bt.s1y1 = f.mul(k.aS1, y1);
  bt.s2y2 = f.mul(k.aS2, y2);
  bt.t1du = f.mul(k.bT1, du);
  bt.t2d2 = f.mul(k.bT2, d2);
  return fma(bt.s1y1, y1, fma(bt.s2y2, y2, fma(bt.t1du, du, fma(bt.t2d2, d2, k.eps))));
}

// Backward of beta0_eps_s from its saved products: given e0b (the adjoint of beta0 + eps), adds
// those of dm, dp, ym, yp.
//   d/dsv = 2 S1 y1, d/ddu = N1 2 S1 y1 + 2 T1 du, d/ddv = 2 S2 y2, d/dd2 = N2 2 S2 y2 + 2 T2 d2.
__device__ __forceinline__ void beta0_eps_s_bwd(const BetaTerms& bt, const AdjK& k, double e0b, double& dmb,
                                                double& dpb, double& ymb, double& ypb, const FU& f) {
  const double e0b2 = f.add(e0b, e0b);  // 2 e0b, exactly
  const double t1 = f.mul(bt.s1y1, e0b2), t2 = f.mul(bt.s2y2, e0b2);
  const double dub = fma(k.aN1, t1, f.mul(bt.t1du, e0b2));
  const double d2b = fma(k.aN2, t2, f.mul(bt.t2d2, e0b2));
  dmb = f.add(dmb, f.sub(dub, d2b));
  dpb = f.add(dpb, f.add(dub, d2b));
  ymb = f.add(ymb, f.add(t1, t2));
  ypb = f.add(ypb, f.sub(t1, t2));
}

// x sgn(s) with sgn(0) = 0, in the integer pipe: the sign bit of s flips that of x, and a zero s
// (either sign) gives +0
__device__ __forceinline__ double mul_sgn(double x, double s) {
  const int sh = __double2hiint(s), sl = __double2loint(s);
  const bool zero = ((sh & 0x7fffffff) | sl) == 0;
  const double y = __hiloint2double(__double2hiint(x) ^ (sh & (int)0x80000000), __double2loint(x));
  return zero ? 0.0 : y;
}

// Backward of weights_e (W_l = P + tau Q_l from e_l = beta_l + eps, tau = (|e0 - e1| + |e0 - e2|)^2
// / 4) with tau saved by the forward pass: given W0b..W2b, adds the adjoints of e0, e1, e2.
__device__ __forceinline__ void weights_e_bwd(double e0, double e1, double e2, double tau, double W0b, double W1b,
                                              double W2b, double& e0b, double& e1b, double& e2b, const FU& f) {
  const double a = f.sub(e0, e1), b = f.sub(e0, e2);
  const double ts = f.add(fabs(a), fabs(b));
  const double Q0 = f.mul(e1, e2), Q1 = f.mul(e0, e2), Q2 = f.mul(e0, e1);
  const double Pb = f.add(f.add(W0b, W1b), W2b);
  const double taub = fma(W0b, Q0, fma(W1b, Q1, f.mul(W2b, Q2)));
  const double Q0b = fma(W0b, tau, f.mul(Pb, e0)), Q1b = f.mul(W1b, tau), Q2b = f.mul(W2b, tau);
  const double tsb = f.mul(0.5 * ts, taub);
  // the adjoint of ts reaches e0 - e1 and e0 - e2 times their signs
  const double ta = mul_sgn(tsb, a), tb = mul_sgn(tsb, b);
  e0b = f.add(e0b, f.add(f.add(ta, tb), fma(Pb, Q0, fma(Q1b, e2, f.mul(Q2b, e1)))));
  e1b = f.add(e1b, f.sub(fma(Q0b, e2, f.mul(Q2b, e0)), ta));
  e2b = f.add(e2b, f.sub(fma(Q0b, e1, f.mul(Q1b, e0)), tb));
}

// ---------------------------------------------------------------------------------------------
// Backward passes from saved forward values.  The adjoint kernels run the forward interpolation
// once, keep each stencil's intermediates (beta0 + eps, the three weights, the candidate
// combination, the weighted sum, 1/den, tau and the four products of the indicator) in shared
// memory, and the backward pass reads them instead of recomputing them.  The forward map is taken in difference form, as the forward kernels
// take it: the characteristic fields enter only through differences of neighbouring cells.  sv
// points at this thread's first slot; consecutive values are `stride` doubles apart (one slot per
// thread of the block).
constexpr int kStencilSaved = 12;                 // per stencil
constexpr int kFaceSaved = 2 * kStencilSaved;     // per characteristic field of a face (two stencils)
constexpr int kCellSaved = kStencilSaved;         // per characteristic field of a cell

// slots 7..11 of a stencil: tau and the indicator's products
__device__ __forceinline__ void save_tail(double* sv, int stride, double tau, const BetaTerms& bt) {
  sv[7 * stride] = tau;
  sv[8 * stride] = bt.s1y1;
  sv[9 * stride] = bt.s2y2;
  sv[10 * stride] = bt.t1du;
  sv[11 * stride] = bt.t2d2;
}
__device__ __forceinline__ BetaTerms load_terms(const double* sv, int stride) {
  return BetaTerms{sv[8 * stride], sv[9 * stride], sv[10 * stride], sv[11 * stride]};
}

// One characteristic field at one face k+1/2 (the forward kernels' face_field_d) from the
// differences d01 = w1 - w0, d12 = w2 - w1, d23 = w3 - w2 of the cells k-1..k+2 and their
// unscaled derivatives y0..y3 along the direction of k: um - w1 and up - w2 (the interface values
// less the centre values; Eqs. Pxi, interp), saving the intermediates [e0, W0, W1, W2, r, X,
// 1/den, tau, S1 y1, S2 y2, T1 du, T2 d2] of the stencil of cell k, then of cell k+1.
__device__ __forceinline__ void face_field_save(double d01, double d12, double d23, double y0, double y1,
                                                double y2, double y3, const AdjK& k, double& dum, double& dup,
                                                double* sv, int stride, const FU& f) {
  const double e01 = fma(d01, d01, k.eps), e12 = fma(d12, d12, k.eps), e23 = fma(d23, d23, k.eps);
  double du, svs;
  BetaTerms bt;
  {
    const double e0 = beta0_eps_s(d01, d12, y0, y2, k, f, du, svs, bt);
    const Wts wt = weights_e(e0, e01, e12, f);
    const double r = fma(k.dm[0], d01, fma(k.dm[1], d12, fma(k.dm[2], y0, f.mul(k.dm[3], y2))));
    const double sl = fma(wt.W1, d01, f.mul(wt.W2, d12));
    const double inv = rcp(fma(k.G, wt.W0, f.add(wt.W1, wt.W2)), f);
    const double X = fma(wt.W0, r, 0.5 * sl);
    dum = f.mul(X, inv);
    sv[0] = e0;
    sv[stride] = wt.W0;
    sv[2 * stride] = wt.W1;
    sv[3 * stride] = wt.W2;
    sv[4 * stride] = r;
    sv[5 * stride] = X;
    sv[6 * stride] = inv;
    save_tail(sv, stride, wt.tau, bt);
  }
  {
    double* const s2 = sv + kStencilSaved * stride;
    const double e0 = beta0_eps_s(d12, d23, y1, y3, k, f, du, svs, bt);
    const Wts wt = weights_e(e0, e12, e23, f);
    const double r = fma(k.dp[0], d12, fma(k.dp[1], d23, fma(k.dp[2], y1, f.mul(k.dp[3], y3))));
    const double sl = fma(wt.W1, d12, f.mul(wt.W2, d23));
    const double inv = rcp(fma(k.G, wt.W0, f.add(wt.W1, wt.W2)), f);
    const double X = fma(wt.W0, r, -0.5 * sl);
    dup = f.mul(X, inv);
    s2[0] = e0;
    s2[stride] = wt.W0;
    s2[2 * stride] = wt.W1;
    s2[3 * stride] = wt.W2;
    s2[4 * stride] = r;
    s2[5 * stride] = X;
    s2[6 * stride] = inv;
    save_tail(s2, stride, wt.tau, bt);
  }
}

// Backward of face_field_save: given the adjoints of um - w1 and up - w2, adds those of d01, d12,
// d23 (db) and y0..y3 (yb).  um - w1 = X / den with X = W0 r + (W1 d01 + W2 d12)/2,
// den = G W0 + W1 + W2 (up - w2 likewise with d12, d23 and -1/2).
__device__ __forceinline__ void face_field_bwd_saved(double d01, double d12, double d23, double y0, double y1,
                                                     double y2, double y3, const AdjK& k, double umb, double upb,
                                                     const double* sv, int stride, double* db, double* yb,
                                                     const FU& f) {
  const double e01 = fma(d01, d01, k.eps), e12 = fma(d12, d12, k.eps), e23 = fma(d23, d23, k.eps);
  double d01b = 0.0, d12b = 0.0, d23b = 0.0, e01b = 0.0, e12b = 0.0, e23b = 0.0;
  {
    const double e0 = sv[0], W0 = sv[stride], W1 = sv[2 * stride], W2 = sv[3 * stride];
    const double r = sv[4 * stride], X = sv[5 * stride], inv = sv[6 * stride];
    const double Xb = f.mul(umb, inv);
    const double denb = f.mul(f.mul(-Xb, X), inv);
    const double hX = 0.5 * Xb;
    const double W0b = fma(Xb, r, f.mul(denb, k.G)), W1b = fma(hX, d01, denb), W2b = fma(hX, d12, denb);
    const double rb = f.mul(Xb, W0);
    d01b = f.add(d01b, fma(k.dm[0], rb, f.mul(hX, W1)));
    d12b = f.add(d12b, fma(k.dm[1], rb, f.mul(hX, W2)));
    yb[0] += k.dm[2] * rb;
    yb[2] += k.dm[3] * rb;
    double e0b = 0.0;
    weights_e_bwd(e0, e01, e12, sv[7 * stride], W0b, W1b, W2b, e0b, e01b, e12b, f);
    beta0_eps_s_bwd(load_terms(sv, stride), k, e0b, d01b, d12b, yb[0], yb[2], f);
  }
  {
    const double* const s2 = sv + kStencilSaved * stride;
    const double e0 = s2[0], W0 = s2[stride], W1 = s2[2 * stride], W2 = s2[3 * stride];
    const double r = s2[4 * stride], X = s2[5 * stride], inv = s2[6 * stride];
    const double Xb = f.mul(upb, inv);
    const double denb = f.mul(f.mul(-Xb, X), inv);
    const double hX = -0.5 * Xb;
    const double W0b = fma(Xb, r, f.mul(denb, k.G)), W1b = fma(hX, d12, denb), W2b = fma(hX, d23, denb);
    const double rb = f.mul(Xb, W0);
    d12b = f.add(d12b, fma(k.dp[0], rb, f.mul(hX, W1)));
    d23b = f.add(d23b, fma(k.dp[1], rb, f.mul(hX, W2)));
    yb[1] += k.dp[2] * rb;
    yb[3] += k.dp[3] * rb;
    double e0b = 0.0;
    weights_e_bwd(e0, e12, e23, s2[7 * stride], W0b, W1b, W2b, e0b, e12b, e23b, f);
    beta0_eps_s_bwd(load_terms(s2, stride), k, e0b, d12b, d23b, yb[1], yb[3], f);
  }
  // e_kl = d_kl^2 + eps
  db[0] = f.add(db[0], fma(2.0 * d01, e01b, d01b));
  db[1] = f.add(db[1], fma(2.0 * d12, e12b, d12b));
  db[2] = f.add(db[2], fma(2.0 * d23, e23b, d23b));
}

// The limiter (Eq. limiter) of one characteristic field from the differences d01 = w1 - w0,
// d12 = w2 - w1 and the unscaled derivatives y0, y2 (the forward kernels' cell_field_d): h v~_i,
// saving [e0, W0, W1, W2, t, num, 1/den, tau, S1 y1, S2 y2, T1 du, T2 d2].
__device__ __forceinline__ double cell_field_save(double d01, double d12, double y0, double y2, const AdjK& k,
                                                  double* sv, int stride, const FU& f) {
  double du, svs;
  BetaTerms bt;
  const double e0 = beta0_eps_s(d01, d12, y0, y2, k, f, du, svs, bt);
  const Wts wt = weights_e(e0, fma(d01, d01, k.eps), fma(d12, d12, k.eps), f);
  const double t = fma(k.cdu, du, -f.mul(k.csv, svs));
  const double num = fma(wt.W0, t, fma(wt.W1, d01, f.mul(wt.W2, d12)));
  const double inv = rcp(fma(k.Gd, wt.W0, f.add(wt.W1, wt.W2)), f);
  sv[0] = e0;
  sv[stride] = wt.W0;
  sv[2 * stride] = wt.W1;
  sv[3 * stride] = wt.W2;
  sv[4 * stride] = t;
  sv[5 * stride] = num;
  sv[6 * stride] = inv;
  save_tail(sv, stride, wt.tau, bt);
  return f.mul(num, inv);
}

// Backward of cell_field_save from its saved values: given the adjoint of its output, adds those
// of d01, d12 (db) and y0, y2.
__device__ __forceinline__ void cell_field_bwd_saved(double d01, double d12, double y0, double y2, const AdjK& k,
                                                     double outb, const double* sv, int stride, double* db,
                                                     double& y0b, double& y2b, const FU& f) {
  const double e1 = fma(d01, d01, k.eps), e2 = fma(d12, d12, k.eps);
  const double e0 = sv[0], W0 = sv[stride], W1 = sv[2 * stride], W2 = sv[3 * stride];
  const double t = sv[4 * stride], num = sv[5 * stride], inv = sv[6 * stride];
  const double numb = f.mul(outb, inv);
  const double denb = f.mul(f.mul(-numb, num), inv);
  const double W0b = fma(numb, t, f.mul(denb, k.Gd)), W1b = fma(numb, d01, denb), W2b = fma(numb, d12, denb);
  const double tb = f.mul(numb, W0);
  double d01b = f.mul(numb, W1), d12b = f.mul(numb, W2);
  // t = cdu (d01 + d12) - csv (y0 + y2), csv = ucsv of the direction
  d01b += k.cdu * tb;
  d12b += k.cdu * tb;
  y0b -= k.csv * tb;
  y2b -= k.csv * tb;
  double e0b = 0.0, e1b = 0.0, e2b = 0.0;
  weights_e_bwd(e0, e1, e2, sv[7 * stride], W0b, W1b, W2b, e0b, e1b, e2b, f);
  beta0_eps_s_bwd(load_terms(sv, stride), k, e0b, d01b, d12b, y0b, y2b, f);
  db[0] = f.add(db[0], fma(2.0 * d01, e1b, d01b));
  db[1] = f.add(db[1], fma(2.0 * d12, e2b, d12b));
}

// ---------------------------------------------------------------------------------------------
// Eigenvector products.  EigBar accumulates the adjoints of the eigen-state variables.
struct EigBar {
  double u, v, H, c, ic;
};

template <int NC>
__device__ __forceinline__ void project_bwd(const Eig<NC>& e, const double* q, const double* wbar, double* qbar,
                                            double& hb1b, double& hb2b, double& hicb, EigBar& eb,
                                            const FU& f = HW_PLAIN_FU) {
  // forward: k, th = hb2 q0 - hb1 k, sh = (u q0 - q1) hic
  const double k = NC == 4 ? f.sub(fma(e.v, q[2], f.mul(e.u, q[1])), q[3]) : fma(e.u, q[1], -q[NC - 1]);
  const double m = fma(e.u, q[0], -q[1]);
  const double wr = NC == 4 ? wbar[3] : wbar[2];
  const double thb = f.add(fma(-2.0, wbar[1], wbar[0]), wr);
  const double shb = f.sub(wbar[0], wr);
  qbar[0] = f.add(qbar[0], wbar[1]);
  if (NC == 4) {
    qbar[0] -= e.v * wbar[2];
    qbar[2] = f.add(qbar[2], wbar[2]);
    eb.v -= wbar[2] * q[0];
  }
  // th
  hb2b += thb * q[0];
  qbar[0] += thb * e.hb2;
  hb1b -= thb * k;
  const double kb = f.mul(-thb, e.hb1);
  // sh
  const double mb = f.mul(shb, e.hic);
  hicb += shb * m;
  eb.u += mb * q[0];
  qbar[0] += mb * e.u;
  qbar[1] = f.sub(qbar[1], mb);
  // k
  eb.u += kb * q[1];
  qbar[1] += kb * e.u;
  if (NC == 4) {
    eb.v += kb * q[2];
    qbar[2] += kb * e.v;
    qbar[3] = f.sub(qbar[3], kb);
  } else {
    qbar[NC - 1] = f.sub(qbar[NC - 1], kb);
  }
}

template <int NC>
__device__ __forceinline__ void back_bwd(const Eig<NC>& e, const double* w, const double* qbar, double* wbar,
                                         double& hq2b, double& ucb, EigBar& eb, const FU& f = HW_PLAIN_FU) {
  const double wl = w[0], wr = NC == 4 ? w[3] : w[2];
  const double sg = f.add(wl, wr), dl = f.sub(wr, wl);
  const double q0 = f.add(sg, w[1]);
  double sgb = 0.0, dlb = 0.0, q0b = qbar[0];
  if (NC == 4) {
    // q3 = H sg + hq2 w1 + v w2 + uc dl
    eb.H += qbar[3] * sg;
    sgb += qbar[3] * e.H;
    hq2b += qbar[3] * w[1];
    wbar[1] += qbar[3] * e.hq2;
    eb.v += qbar[3] * w[2];
    wbar[2] += qbar[3] * e.v;
    ucb += qbar[3] * dl;
    dlb += qbar[3] * e.uc;
    // q2 = v q0 + w2
    eb.v += qbar[2] * q0;
    q0b += qbar[2] * e.v;
    wbar[2] = f.add(wbar[2], qbar[2]);
  } else {
    // q2 = H sg + hq2 w1 + uc dl
    eb.H += qbar[2] * sg;
    sgb += qbar[2] * e.H;
    hq2b += qbar[2] * w[1];
    wbar[1] += qbar[2] * e.hq2;
    ucb += qbar[2] * dl;
    dlb += qbar[2] * e.uc;
  }
  // q1 = u q0 + c dl
  eb.u += qbar[1] * q0;
  q0b += qbar[1] * e.u;
  eb.c += qbar[1] * dl;
  dlb += qbar[1] * e.c;
  // q0 = sg + w1
  sgb = f.add(sgb, q0b);
  wbar[1] = f.add(wbar[1], q0b);
  wbar[0] = f.add(wbar[0], f.sub(sgb, dlb));
  if (NC == 4)
    wbar[3] = f.add(wbar[3], f.add(sgb, dlb));
  else
    wbar[2] = f.add(wbar[2], f.add(sgb, dlb));
}

// adjoints of the derived eigen quantities (hb1, hb2, hic, hq2, uc) into (u, v, c, ic)
template <int NC>
__device__ __forceinline__ void setup_bwd(const Eig<NC>& e, double gm1, double ic, double hb1b, double hb2b,
                                          double hicb, double hq2b, double ucb, EigBar& eb) {
  // hb2 = hb1 hq2
  hb1b += hb2b * e.hq2;
  hq2b += hb2b * e.hb1;
  // hb1 = gm1 ic^2 / 2
  eb.ic += hb1b * gm1 * ic;
  // hic = ic / 2
  eb.ic += 0.5 * hicb;
  // hq2 = (u^2 + v^2) / 2
  eb.u += hq2b * e.u;
  if (NC == 4) eb.v += hq2b * e.v;
  // uc = u c
  eb.u += ucb * e.c;
  eb.c += ucb * e.u;
}

// ---------------------------------------------------------------------------------------------
// Euler primitives of one cell in the normal frame, for the backward routines.
template <int NC>
struct Prim {
  double ir, u, v, p;
};

template <int NC>
__device__ __forceinline__ Prim<NC> prim_of(const double* U, double gm1, const FU& f = HW_PLAIN_FU) {
  Prim<NC> q;
  q.ir = rcp(U[0], f);
  q.u = f.mul(U[1], q.ir);
  q.v = NC == 4 ? f.mul(U[2], q.ir) : 0.0;
  const double ke = NC == 4 ? fma(U[1], q.u, f.mul(U[2], q.v)) : f.mul(U[1], q.u);
  q.p = gm1 * fma(-0.5, ke, U[NC - 1]);
  return q;
}

// Given the adjoints of (ir, u, v, p) of a cell, adds those of U.
template <int NC>
__device__ __forceinline__ void prim_bwd(const double* U, const Prim<NC>& q, double gm1, double irb, double ub,
                                         double vb, double pb, double* Ub, const FU& f = HW_PLAIN_FU) {
  // p = gm1 (E - (m u + n v)/2)
  Ub[NC - 1] += gm1 * pb;
  const double keb = -0.5 * gm1 * pb;
  Ub[1] += keb * q.u;
  ub += keb * U[1];
  if (NC == 4) {
    Ub[2] += keb * q.v;
    vb += keb * U[2];
  }
  // u = m ir, v = n ir
  Ub[1] += ub * q.ir;
  irb += ub * U[1];
  if (NC == 4) {
    Ub[2] += vb * q.ir;
    irb += vb * U[2];
  }
  // ir = 1/rho
  Ub[0] = fma(-f.mul(irb, q.ir), q.ir, Ub[0]);
}

// Flux F(U) in the normal frame: given Fb, adds Ub.  q: the primitives of U (prim_of).
template <int NC>
__device__ __forceinline__ void flux_bwd(const double* U, const Prim<NC>& q, double gm1, const double* Fb, double* Ub,
                                         const FU& f = HW_PLAIN_FU) {
  double ub = 0.0, vb = 0.0, pb = 0.0;
  // F = (m, m u + p, [n u,] (E + p) u)
  Ub[1] = f.add(Ub[1], fma(Fb[1], q.u, Fb[0]));
  ub += Fb[1] * U[1];
  pb += Fb[1];
  if (NC == 4) {
    Ub[2] += Fb[2] * q.u;
    ub += Fb[2] * U[2];
  }
  Ub[NC - 1] += Fb[NC - 1] * q.u;
  pb += Fb[NC - 1] * q.u;
  ub += Fb[NC - 1] * f.add(U[NC - 1], q.p);
  prim_bwd<NC>(U, q, gm1, 0.0, ub, vb, pb, Ub, f);
}

// Jacobian product A(U) D in the normal frame: given ob, adds Ub and Db.  q: the primitives of U.
template <int NC>
__device__ __forceinline__ void jvp_bwd(const double* U, const Prim<NC>& q, const double* D, double gm1,
                                        const double* ob, double* Ub, double* Db, const FU& f = HW_PLAIN_FU) {
  const double du = f.mul(fma(-q.u, D[0], D[1]), q.ir);
  const double dv = NC == 4 ? f.mul(fma(-q.v, D[0], D[2]), q.ir) : 0.0;
  const double dk = NC == 4 ? fma(D[1], q.u, fma(U[1], du, fma(D[2], q.v, f.mul(U[2], dv))))
                            : fma(D[1], q.u, f.mul(U[1], du));
  const double dp = gm1 * fma(-0.5, dk, D[NC - 1]);
  double ub = 0.0, vb = 0.0, pb = 0.0, irb = 0.0, dub = 0.0, dvb = 0.0, dpb = 0.0;
  // out0 = D1
  Db[1] = f.add(Db[1], ob[0]);
  // out1 = D1 u + m du + dp
  Db[1] += ob[1] * q.u;
  ub += ob[1] * D[1];
  Ub[1] += ob[1] * du;
  dub += ob[1] * U[1];
  dpb = f.add(dpb, ob[1]);
  if (NC == 4) {
    // out2 = D2 u + n du
    Db[2] += ob[2] * q.u;
    ub += ob[2] * D[2];
    Ub[2] += ob[2] * du;
    dub += ob[2] * U[2];
  }
  // out_last = (D_E + dp) u + (E + p) du
  Db[NC - 1] += ob[NC - 1] * q.u;
  dpb += ob[NC - 1] * q.u;
  ub += ob[NC - 1] * f.add(D[NC - 1], dp);
  Ub[NC - 1] += ob[NC - 1] * du;
  pb += ob[NC - 1] * du;
  dub += ob[NC - 1] * f.add(U[NC - 1], q.p);
  // dp = gm1 (D_E - dk/2)
  Db[NC - 1] += gm1 * dpb;
  const double dkb = -0.5 * gm1 * dpb;
  // dk = D1 u + m du [+ D2 v + n dv]
  Db[1] += dkb * q.u;
  ub += dkb * D[1];
  Ub[1] += dkb * du;
  dub += dkb * U[1];
  if (NC == 4) {
    Db[2] += dkb * q.v;
    vb += dkb * D[2];
    Ub[2] += dkb * dv;
    dvb += dkb * U[2];
  }
  // du = (D1 - u D0) ir, dv = (D2 - v D0) ir
  Db[1] += dub * q.ir;
  ub = fma(-f.mul(dub, D[0]), q.ir, ub);
  Db[0] = fma(-f.mul(dub, q.u), q.ir, Db[0]);
  irb += dub * fma(-q.u, D[0], D[1]);
  if (NC == 4) {
    Db[2] += dvb * q.ir;
    vb = fma(-f.mul(dvb, D[0]), q.ir, vb);
    Db[0] = fma(-f.mul(dvb, q.v), q.ir, Db[0]);
    irb += dvb * fma(-q.v, D[0], D[2]);
  }
  prim_bwd<NC>(U, q, gm1, irb, ub, vb, pb, Ub, f);
}

}  // namespace hw
