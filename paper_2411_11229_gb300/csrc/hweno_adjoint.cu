// Adjoint of one SSP-RK3 step of the Euler equations (1D and 2D), hand-written: see
// include/hweno.h (hweno_adjoint_step) for the contract.
//
// The vector-Jacobian product of one stage operator, lam = (dM/dS)^T muM + (dL/dS)^T muL at a
// stage input S with alpha fixed, is the transpose of the forward kernels:
//   k_adj_cell   per cell and direction: backward of the modified derivative (Eq. limiter in the
//                cell's characteristic fields): contributions to U of cells i-1..i+1 and to the
//                derivative of cells i-1, i+1;
//   k_adj_face   per face: recomputes the face and back-propagates the flux adjoint
//                nu = (muL[right cell] - muL[left cell]) / h through the LF fluxes at U^+-, the
//                back projection, the HWENO weights and smoothness indicators, the projections,
//                the eigenvectors and the Roe average: contributions to U and to the derivative
//                of the four cells of the face;
//   k_adj_gather per cell: collects those contributions, applies the transposes of the (linear)
//                D-terms and mixed fluxes to the flux adjoints and the nodal flux VJPs, and adds
//                the identity part of M.
// Contributions are stored per face / per cell and gathered (no atomics: deterministic).
#include <cmath>
#include "hweno_adjoint.cuh"
#include "hweno_host.cuh"

using namespace hwh;

namespace hw {

struct AdjWork {
  double* CU;  // face contributions to U: [dir][face][4 cells][NC] (original frame)
  double* CD;  // face contributions to the own-direction derivative, same layout
  double* CM;  // modified-derivative contributions: [dir][cell][3 U + 2 D][NC] (original frame)
  const double* scal;  // the handle's scalars; [4..7] are zero (read by fu_of)
};

template <int DIM>
__device__ __forceinline__ long long nfaces_dir(const Grid& g, int dir) {
  return dir == 0 ? (long long)(g.nx + 1) * g.ny : (long long)(g.ny + 1) * g.nx;
}

// -------------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_adj_cell(Grid g, const double* __restrict__ S, const double* __restrict__ muM,
                                                       AdjWork aw) {
  constexpr int NC = DIM == 1 ? 3 : 4;
  const int d = blockIdx.y;
  const long long plane = g.plane;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= plane) return;
  const int i = (int)(p % g.nx), j = (int)(p / g.nx);
  const int n = d == 0 ? g.nx : g.ny;
  const int a0 = d == 0 ? i : j;
  const int fld = d == 0 ? 1 : 2;
  const double ih = g.ih[d];
  const FU fu = fu_of(aw.scal);
  // the derivatives enter unscaled, as in the forward cell kernel (h folded into the constants)
  double U3[3][NC], D3[3][NC];
  long long pc[3];
  bool refl[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int ac = bc_map(a0 - 1 + q, n, g.bc, refl[q]);
    pc[q] = HW_IDX(d == 0 ? (long long)j * g.nx + ac : (long long)ac * g.nx + i, plane);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      U3[q][k] = S[k * plane + pc[q]];
      D3[q][k] = S[(fld * NC + k) * plane + pc[q]];
    }
    if (d == 1) {
      swap_frame<NC>(U3[q]);
      swap_frame<NC>(D3[q]);
    }
    mirror_U<NC>(U3[q], refl[q]);
    mirror_D<NC>(D3[q], refl[q]);
  }
  // forward: eigenvectors of the cell's own state
  const Prim<NC> pr = prim_of<NC>(U3[1], g.gm1, fu);
  const double H = (U3[1][NC - 1] + pr.p) * pr.ir;
  const double c2 = g.gamma * pr.p * pr.ir;
  const double ic = rsqrt(c2);
  const double c = c2 * ic;
  Eig<NC> e;
  e.setup(pr.u, pr.v, H, c, ic, g.gm1);
  // the limiter sees the characteristic fields only through differences of neighbouring cells
  double dU[2][NC], Dq[2][NC], Zm[NC], Zp[NC], ht[NC];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < NC; ++k) dU[q][k] = fu.sub(U3[q + 1][k], U3[q][k]);
  e.project(dU[0], Dq[0], fu);
  e.project(dU[1], Dq[1], fu);
  e.project(D3[0], Zm, fu);
  e.project(D3[2], Zp, fu);
  // forward intermediates of the limiter, per field, kept in this thread's shared-memory slots
  extern __shared__ double adj_cell_sm[];
  double* const svb = adj_cell_sm + threadIdx.x;
  const AdjK ak = adj_k(g, d, fu);
#pragma unroll
  for (int s = 0; s < NC; ++s)
    ht[s] = cell_field_save(Dq[0][s], Dq[1][s], Zm[s], Zp[s], ak, svb + s * kCellSaved * kThreads, kThreads, fu) * ih;
  // backward from the adjoint of the modified derivative of this cell
  double ob[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) ob[k] = muM[(fld * NC + k) * plane + p];
  if (d == 1) swap_frame<NC>(ob);
  EigBar eb = {0.0, 0.0, 0.0, 0.0, 0.0};
  double hq2b = 0.0, ucb = 0.0, hb1b = 0.0, hb2b = 0.0, hicb = 0.0;
  double htb[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) htb[s] = 0.0;
  back_bwd<NC>(e, ht, ob, htb, hq2b, ucb, eb, fu);
  double Dqb[2][NC], Zmb[NC], Zpb[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    double db[2] = {0.0, 0.0};
    Zmb[s] = Zpb[s] = 0.0;
    cell_field_bwd_saved(Dq[0][s], Dq[1][s], Zm[s], Zp[s], ak, htb[s] * ih, svb + s * kCellSaved * kThreads,
                         kThreads, db, Zmb[s], Zpb[s], fu);
    Dqb[0][s] = db[0];
    Dqb[1][s] = db[1];
  }
  double dUb[2][NC], Ub[3][NC], Dmb[NC], Dpb[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    dUb[0][k] = dUb[1][k] = 0.0;
    Dmb[k] = Dpb[k] = 0.0;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) project_bwd<NC>(e, dU[q], Dqb[q], dUb[q], hb1b, hb2b, hicb, eb, fu);
  project_bwd<NC>(e, D3[0], Zmb, Dmb, hb1b, hb2b, hicb, eb, fu);
  project_bwd<NC>(e, D3[2], Zpb, Dpb, hb1b, hb2b, hicb, eb, fu);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    Ub[0][k] = -dUb[0][k];
    Ub[1][k] = fu.sub(dUb[0][k], dUb[1][k]);
    Ub[2][k] = dUb[1][k];
  }
  setup_bwd<NC>(e, g.gm1, ic, hb1b, hb2b, hicb, hq2b, ucb, eb);
  // c = sqrt(c2), ic = 1/sqrt(c2), c2 = gamma p ir, H = (E + p) ir
  const double c2b = 0.5 * ic * (eb.c - eb.ic * ic * ic);
  double pb = c2b * g.gamma * pr.ir + eb.H * pr.ir;
  double irb = c2b * g.gamma * pr.p + eb.H * (U3[1][NC - 1] + pr.p);
  Ub[1][NC - 1] += eb.H * pr.ir;
  prim_bwd<NC>(U3[1], pr, g.gm1, irb, eb.u, eb.v, pb, Ub[1], fu);
  // a mirrored neighbour was read through the sign table: its contributions go back through it
  // (the table is its own transpose)
#pragma unroll
  for (int q = 0; q < 3; ++q) mirror_U<NC>(Ub[q], refl[q]);
  mirror_D<NC>(Dmb, refl[0]);
  mirror_D<NC>(Dpb, refl[2]);
  // store (original frame): 3 U contributions, then the derivative adjoints of cells i-1, i+1
  double* out = aw.CM + ((long long)d * plane + p) * 5 * NC;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (d == 1) swap_frame<NC>(Ub[q]);
#pragma unroll
    for (int k = 0; k < NC; ++k) out[q * NC + k] = Ub[q][k];
  }
  if (d == 1) {
    swap_frame<NC>(Dmb);
    swap_frame<NC>(Dpb);
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    out[3 * NC + k] = Dmb[k];
    out[4 * NC + k] = Dpb[k];
  }
}

// -------------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_adj_face(Grid g, const double* __restrict__ S, const double* __restrict__ muL,
                                                       AdjWork aw, const double* __restrict__ alpha2) {
  constexpr int NC = DIM == 1 ? 3 : 4;
  const int dir = blockIdx.y;
  const long long plane = g.plane;
  const int n = dir == 0 ? g.nx : g.ny;
  const int nlines = dir == 0 ? g.ny : g.nx;
  const long long f = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (f >= (long long)(n + 1) * nlines) return;
  int fa, line;
  if (dir == 0) {
    line = (int)(f / (n + 1));
    fa = (int)(f % (n + 1));
  } else {
    fa = (int)(f / g.nx);
    line = (int)(f % g.nx);
  }
  long long pc[4];
  bool refl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = bc_map(fa - 2 + q, n, g.bc, refl[q]);
    pc[q] = HW_IDX(dir == 0 ? (long long)line * g.nx + a : (long long)a * g.nx + line, plane);
  }
  const int fown = dir == 0 ? 1 : 2;
  // 1/(2h): the flux adjoints below are differences (mu_L[right] - mu_L[left]) without their 1/h,
  // which this coefficient carries together with the 1/2 of the LF fluxes
  const double hih = g.hih[dir];
  const double k21 = g.uvd[dir][0], k3 = g.uvd[dir][1];
  const double alpha = alpha2[dir];
  const FU fu = fu_of(aw.scal);
  double Uq[4][NC], Zq[4][NC];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Uq[q][k] = S[k * plane + pc[q]];
      Zq[q][k] = S[(fown * NC + k) * plane + pc[q]];  // unscaled, as in the forward face kernel
    }
    if (dir == 1) {
      swap_frame<NC>(Uq[q]);
      swap_frame<NC>(Zq[q]);
    }
    mirror_U<NC>(Uq[q], refl[q]);
    mirror_D<NC>(Zq[q], refl[q]);
  }
  // adjoints of the face fluxes of U and of the own derivative (normal frame)
  double nuf[NC], nuh[NC];
  {
    const bool hasL = fa - 1 >= 0, hasR = fa <= n - 1;
    const long long cL = dir == 0 ? (long long)line * g.nx + (fa - 1) : (long long)(fa - 1) * g.nx + line;
    const long long cR = dir == 0 ? (long long)line * g.nx + fa : (long long)fa * g.nx + line;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const double rf = hasR ? muL[k * plane + HW_IDX(cR, plane)] : 0.0;
      const double lf = hasL ? muL[k * plane + HW_IDX(cL, plane)] : 0.0;
      const double rh = hasR ? muL[(fown * NC + k) * plane + HW_IDX(cR, plane)] : 0.0;
      const double lh = hasL ? muL[(fown * NC + k) * plane + HW_IDX(cL, plane)] : 0.0;
      nuf[k] = fu.sub(rf, lf);
      nuh[k] = fu.sub(rh, lh);
    }
    if (dir == 1) {
      swap_frame<NC>(nuf);
      swap_frame<NC>(nuh);
    }
  }
  // ---- forward recomputation
  const Prim<NC> pl = prim_of<NC>(Uq[1], g.gm1, fu), prr = prim_of<NC>(Uq[2], g.gm1, fu);
  const double sl = sqrt(Uq[1][0]), sr = sqrt(Uq[2][0]);
  const double Hl = (Uq[1][NC - 1] + pl.p) * pl.ir, Hr = (Uq[2][NC - 1] + prr.p) * prr.ir;
  const double iw = rcp(fu.add(sl, sr), fu);
  const double ub = fu.mul(fma(sl, pl.u, fu.mul(sr, prr.u)), iw);
  const double vb = NC == 4 ? fu.mul(fma(sl, pl.v, fu.mul(sr, prr.v)), iw) : 0.0;
  const double Hb = fu.mul(fma(sl, Hl, fu.mul(sr, Hr)), iw);
  const double c2 = g.gm1 * fma(-0.5, NC == 4 ? fma(ub, ub, vb * vb) : ub * ub, Hb);
  const double ic = rsqrt(c2);
  Eig<NC> e;
  e.setup(ub, vb, Hb, c2 * ic, ic, g.gm1);
  // the interpolation sees the characteristic fields only through differences of neighbouring
  // cells; the interface derivatives (Eq. P'xi) are linear in the stencil and formed in conserved
  // variables (k21 = 21/(16 h), k3 = 3/(16 h))
  double dU[3][NC], Dm[NC], Dp[NC];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int k = 0; k < NC; ++k) dU[q][k] = fu.sub(Uq[q + 1][k], Uq[q][k]);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    Dm[k] = fma(k21, dU[1][k], fma(-k3, dU[0][k], fma(0.0625, Zq[0][k], -0.1875 * Zq[2][k])));
    Dp[k] = fma(k21, dU[1][k], fma(-k3, dU[2][k], fma(-0.1875, Zq[1][k], 0.0625 * Zq[3][k])));
  }
  double Dq[3][NC], Yq[4][NC];
#pragma unroll
  for (int q = 0; q < 3; ++q) e.project(dU[q], Dq[q], fu);
#pragma unroll
  for (int q = 0; q < 4; ++q) e.project(Zq[q], Yq[q], fu);
  double cm[NC], cp[NC];
  // forward intermediates of the interpolation, per field, kept in this thread's shared-memory slots
  extern __shared__ double adj_face_sm[];
  double* const svb = adj_face_sm + threadIdx.x;
  const AdjK ak = adj_k(g, dir, fu);
#pragma unroll
  for (int s = 0; s < NC; ++s)
    face_field_save(Dq[0][s], Dq[1][s], Dq[2][s], Yq[0][s], Yq[1][s], Yq[2][s], Yq[3][s], ak, cm[s], cp[s],
                    svb + s * kFaceSaved * kThreads, kThreads, fu);
  // interface states: centre states plus the back-projected corrections
  double Um[NC], Up[NC];
  e.back_add(cm, Uq[1], Um, fu);
  e.back_add(cp, Uq[2], Up, fu);
  // ---- backward: fh = (FUm + FUp - alpha (Up - Um)) / 2 + Df, hh = (HDm + HDp - alpha (Dp - Dm)) / 2
  // + Dh, with the flux adjoints nuf / h and nuh / h
  double Umb[NC], Upb[NC], Dmb[NC], Dpb[NC], Fb[NC], Hb2[NC];
  const double ha = hih * alpha;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    Umb[k] = ha * nuf[k];
    Upb[k] = -Umb[k];
    Dmb[k] = ha * nuh[k];
    Dpb[k] = -Dmb[k];
    Fb[k] = hih * nuf[k];
    Hb2[k] = hih * nuh[k];
  }
  {
    // the primitives of each interface state, shared by its flux and Jacobian-product backward
    const Prim<NC> qm = prim_of<NC>(Um, g.gm1, fu), qp = prim_of<NC>(Up, g.gm1, fu);
    flux_bwd<NC>(Um, qm, g.gm1, Fb, Umb, fu);
    flux_bwd<NC>(Up, qp, g.gm1, Fb, Upb, fu);
    jvp_bwd<NC>(Um, qm, Dm, g.gm1, Hb2, Umb, Dmb, fu);
    jvp_bwd<NC>(Up, qp, Dp, g.gm1, Hb2, Upb, Dpb, fu);
  }
  EigBar eb = {0.0, 0.0, 0.0, 0.0, 0.0};
  double hq2b = 0.0, ucb = 0.0, hb1b = 0.0, hb2b = 0.0, hicb = 0.0;
  double cmb[NC], cpb[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) cmb[s] = cpb[s] = 0.0;
  back_bwd<NC>(e, cm, Umb, cmb, hq2b, ucb, eb, fu);
  back_bwd<NC>(e, cp, Upb, cpb, hq2b, ucb, eb, fu);
  double Uqb[4][NC], Zqb[4][NC], dUb[3][NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    // the centre states enter Um, Up directly; the derivatives linearly
    Uqb[0][k] = Uqb[3][k] = 0.0;
    Uqb[1][k] = Umb[k];
    Uqb[2][k] = Upb[k];
    dUb[0][k] = -k3 * Dmb[k];
    dUb[1][k] = k21 * fu.add(Dmb[k], Dpb[k]);
    dUb[2][k] = -k3 * Dpb[k];
    Zqb[0][k] = 0.0625 * Dmb[k];
    Zqb[1][k] = -0.1875 * Dpb[k];
    Zqb[2][k] = -0.1875 * Dmb[k];
    Zqb[3][k] = 0.0625 * Dpb[k];
  }
  double Dqb[3][NC], Yb[4][NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    double db[3] = {0.0, 0.0, 0.0}, yb[4] = {0.0, 0.0, 0.0, 0.0};
    face_field_bwd_saved(Dq[0][s], Dq[1][s], Dq[2][s], Yq[0][s], Yq[1][s], Yq[2][s], Yq[3][s], ak, cmb[s], cpb[s],
                         svb + s * kFaceSaved * kThreads, kThreads, db, yb, fu);
#pragma unroll
    for (int q = 0; q < 3; ++q) Dqb[q][s] = db[q];
#pragma unroll
    for (int q = 0; q < 4; ++q) Yb[q][s] = yb[q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) project_bwd<NC>(e, dU[q], Dqb[q], dUb[q], hb1b, hb2b, hicb, eb, fu);
#pragma unroll
  for (int q = 0; q < 4; ++q) project_bwd<NC>(e, Zq[q], Yb[q], Zqb[q], hb1b, hb2b, hicb, eb, fu);
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Uqb[q + 1][k] = fu.add(Uqb[q + 1][k], dUb[q][k]);
      Uqb[q][k] = fu.sub(Uqb[q][k], dUb[q][k]);
    }
  setup_bwd<NC>(e, g.gm1, ic, hb1b, hb2b, hicb, hq2b, ucb, eb);
  // c = sqrt(c2), ic = 1/sqrt(c2); c2 = gm1 (Hb - (ub^2 + vb^2)/2)
  const double c2b = 0.5 * ic * (eb.c - eb.ic * ic * ic);
  const double Hbb = eb.H + g.gm1 * c2b;
  const double ubb = eb.u - g.gm1 * ub * c2b;
  const double vbb = eb.v - g.gm1 * vb * c2b;
  // Roe average: x_b = (sl x_l + sr x_r) iw for x in (u, v, H)
  const double iwb = ubb * fma(sl, pl.u, sr * prr.u) + (NC == 4 ? vbb * fma(sl, pl.v, sr * prr.v) : 0.0) +
                     Hbb * fma(sl, Hl, sr * Hr);
  const double slb = iw * (ubb * pl.u + (NC == 4 ? vbb * pl.v : 0.0) + Hbb * Hl) - iwb * iw * iw;
  const double srb = iw * (ubb * prr.u + (NC == 4 ? vbb * prr.v : 0.0) + Hbb * Hr) - iwb * iw * iw;
  // cells 1 and 2: sqrt(rho), u, v, H = (E + p) ir; d sqrt(rho) / d rho = sqrt(rho) ir / 2
  {
    const double Hlb = Hbb * sl * iw;
    Uqb[1][0] += slb * (0.5 * sl) * pl.ir;
    Uqb[1][NC - 1] += Hlb * pl.ir;
    prim_bwd<NC>(Uq[1], pl, g.gm1, Hlb * (Uq[1][NC - 1] + pl.p), ubb * sl * iw, vbb * sl * iw, Hlb * pl.ir, Uqb[1]);
    const double Hrb = Hbb * sr * iw;
    Uqb[2][0] += srb * (0.5 * sr) * prr.ir;
    Uqb[2][NC - 1] += Hrb * prr.ir;
    prim_bwd<NC>(Uq[2], prr, g.gm1, Hrb * (Uq[2][NC - 1] + prr.p), ubb * sr * iw, vbb * sr * iw, Hrb * prr.ir,
                 Uqb[2]);
  }
  // store (original frame): the contributions to U and to the unscaled derivative of the direction
  const long long fo = HW_IDX(dir == 0 ? (long long)line * (g.nx + 1) + fa : (long long)fa * g.nx + line,
                              dir == 0 ? (long long)(g.nx + 1) * g.ny : (long long)(g.ny + 1) * g.nx);
  const long long base = ((dir == 0 ? 0 : (long long)(g.nx + 1) * g.ny) + fo) * 4 * NC;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    mirror_U<NC>(Uqb[q], refl[q]);
    mirror_D<NC>(Zqb[q], refl[q]);
    if (dir == 1) {
      swap_frame<NC>(Uqb[q]);
      swap_frame<NC>(Zqb[q]);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      aw.CU[base + q * NC + k] = Uqb[q][k];
      aw.CD[base + q * NC + k] = Zqb[q][k];
    }
  }
}

// -------------------------------------------------------------------------------------------
// aliases of cell a (0 <= a < n) among the unmapped indices -2 .. n+1 of the stencils
__device__ __forceinline__ int aliases(int a, int n, int bc, int* x) {
  int k = 0;
  x[k++] = a;
  if (bc == BC_PERIODIC) {
    if (a + n <= n + 1) x[k++] = a + n;
    if (a - n >= -2) x[k++] = a - n;
  } else if (bc == BC_REFLECTIVE) {
    // ghost -1-a mirrors cell a (a = 0, 1), ghost 2n-1-a mirrors it (a = n-1, n-2)
    if (-1 - a >= -2) x[k++] = -1 - a;
    if (2 * n - 1 - a <= n + 1) x[k++] = 2 * n - 1 - a;
  } else {
    if (a == 0) {
      x[k++] = -1;
      x[k++] = -2;
    }
    if (a == n - 1) {
      x[k++] = n;
      x[k++] = n + 1;
    }
  }
  return k;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads, 4) k_adj_gather(Grid g, const double* __restrict__ S,
                                                         const double* __restrict__ muM, const double* __restrict__ muL,
                                                         AdjWork aw, double* __restrict__ lam) {
  constexpr int NC = DIM == 1 ? 3 : 4;
  constexpr int NF = DIM + 1;
  const long long plane = g.plane;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= plane) return;
  const FU fu = fu_of(aw.scal);
  const int i = (int)(p % g.nx), j = (int)(p / g.nx);
  double lb[NF][NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    lb[0][k] = muM[k * plane + p];  // M = (U, ...): identity part
#pragma unroll
    for (int f = 1; f < NF; ++f) lb[f][k] = 0.0;
  }
  double U[NC], V[NF - 1][NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    U[k] = S[k * plane + p];
#pragma unroll
    for (int f = 1; f < NF; ++f) V[f - 1][k] = S[(f * NC + k) * plane + p];
  }
  const Prim<NC> qc = prim_of<NC>(U, g.gm1, fu);  // original frame
  const long long oplx = (long long)g.ny * (g.nx + 1);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int n = d == 0 ? g.nx : g.ny;
    const int a0 = d == 0 ? i : j;
    const int fown = d == 0 ? 1 : 2, foth = d == 0 ? 2 : 1;
    const double ih = g.ih[d];
    int xs[3];
    const int nx_ = aliases(a0, n, g.bc, xs);
    double nf[NC], nh[NC], no[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) nf[k] = nh[k] = no[k] = 0.0;
    // the normal momentum (original frame) and the nodal sign tables of a mirrored alias: f and
    // the mixed value change sign except for the normal momentum, h only for it
    const int km = d == 0 ? 1 : 2;
    const double cf_ih = DCoef::cf * ih, ef_ih = g.efih[d] * ih, eg_ih = g.egih[d] * ih;
    const double ch_ih = g.chh[d] * ih, eh_ih = DCoef::eh * ih;
    const double m7_ih = (7.0 / 12.0) * ih, m1_ih = (-1.0 / 12.0) * ih;
    for (int t = 0; t < nx_; ++t) {
      const int x = xs[t];
      const bool mir = g.bc == BC_REFLECTIVE && (x < 0 || x >= n);
      // faces fa = x + 2 - q hold this cell at position q
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int fa = x + 2 - q;
        if (fa < 0 || fa > n) continue;
        const int line = d == 0 ? j : i;
        const long long fo = HW_IDX(d == 0 ? (long long)line * (g.nx + 1) + fa : (long long)fa * g.nx + line,
                                    d == 0 ? oplx : (long long)(g.ny + 1) * g.nx);
        const long long base = ((d == 0 ? 0 : oplx) + fo) * 4 * NC + q * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          lb[0][k] = fu.add(lb[0][k], aw.CU[base + k]);
          lb[fown][k] = fu.add(lb[fown][k], aw.CD[base + k]);
        }
        // flux adjoints of this face, for the nodal values (D-terms, mixed flux)
        const bool hasL = fa - 1 >= 0, hasR = fa <= n - 1;
        const long long cL = d == 0 ? (long long)line * g.nx + (fa - 1) : (long long)(fa - 1) * g.nx + line;
        const long long cR = d == 0 ? (long long)line * g.nx + fa : (long long)fa * g.nx + line;
        // the transposed D-term and mixed-flux coefficients of position q, with the 1/h of the flux
        // adjoints folded in (only the outer positions carry h in Eq. Cd-1)
        const double s1 = (q == 0 || q == 3) ? cf_ih : -cf_ih;
        const double sdh = q == 0 ? ef_ih : (q == 1 ? -eg_ih : (q == 2 ? eg_ih : -ef_ih));
        const double mq = (q == 1 || q == 2) ? m7_ih : m1_ih;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          auto dmu = [&](int fld) {
            const double r = hasR ? muL[(fld * NC + k) * plane + HW_IDX(cR, plane)] : 0.0;
            const double l = hasL ? muL[(fld * NC + k) * plane + HW_IDX(cL, plane)] : 0.0;
            return fu.sub(r, l);
          };
          // a mirrored alias takes the nodal sign tables: f and the mixed value flip except for the
          // normal momentum, h only for it (sign flips in the integer pipe)
          const bool flip_f = mir && k != km, flip_h = mir && k == km;
          const double nfh = dmu(0), nhh = dmu(fown);
          nf[k] = fma(s1, neg_if(nfh, flip_f), fma(sdh, neg_if(nhh, flip_f), nf[k]));
          if (q == 0 || q == 3)
            nh[k] = fma(q == 0 ? ch_ih : -ch_ih, neg_if(nfh, flip_h), fma(eh_ih, neg_if(nhh, flip_h), nh[k]));
          if (DIM == 2) no[k] = fma(mq, neg_if(dmu(foth), flip_f), no[k]);
        }
      }
      // modified derivatives of cells c = x + 1 - q hold this cell at stencil position q
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int c = x + 1 - q;
        if (c < 0 || c > n - 1) continue;
        const long long pcl = HW_IDX(d == 0 ? (long long)j * g.nx + c : (long long)c * g.nx + i, plane);
        const double* cm = aw.CM + ((long long)d * plane + pcl) * 5 * NC;
#pragma unroll
        for (int k = 0; k < NC; ++k) lb[0][k] = fu.add(lb[0][k], cm[q * NC + k]);
        if (q == 0) {
#pragma unroll
          for (int k = 0; k < NC; ++k) lb[fown][k] = fu.add(lb[fown][k], cm[3 * NC + k]);
        } else if (q == 2) {
#pragma unroll
          for (int k = 0; k < NC; ++k) lb[fown][k] = fu.add(lb[fown][k], cm[4 * NC + k]);
        }
      }
    }
    // nodal VJPs at this cell (normal frame): f(U), A(U) D_own, A(U) D_other
    double Un[NC], Dn[NC], On[NC], Ub[NC], Db[NC], Ob[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Un[k] = U[k];
      Dn[k] = V[fown - 1][k];
      On[k] = DIM == 2 ? V[foth - 1][k] : 0.0;
      Ub[k] = Db[k] = Ob[k] = 0.0;
    }
    if (d == 1) {
      swap_frame<NC>(Un);
      swap_frame<NC>(Dn);
      swap_frame<NC>(On);
      swap_frame<NC>(nf);
      swap_frame<NC>(nh);
      swap_frame<NC>(no);
    }
    // the cell's primitives in the direction's frame (the velocities exchanged in y), shared by
    // the three nodal backward passes and computed once for both directions
    Prim<NC> qn = qc;
    if (d == 1) {
      qn.u = qc.v;
      qn.v = qc.u;
    }
    flux_bwd<NC>(Un, qn, g.gm1, nf, Ub, fu);
    jvp_bwd<NC>(Un, qn, Dn, g.gm1, nh, Ub, Db, fu);
    if (DIM == 2) jvp_bwd<NC>(Un, qn, On, g.gm1, no, Ub, Ob, fu);
    if (d == 1) {
      swap_frame<NC>(Ub);
      swap_frame<NC>(Db);
      swap_frame<NC>(Ob);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      lb[0][k] = fu.add(lb[0][k], Ub[k]);
      lb[fown][k] = fu.add(lb[fown][k], Db[k]);
      if (DIM == 2) lb[foth][k] = fu.add(lb[foth][k], Ob[k]);
    }
  }
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int k = 0; k < NC; ++k) lam[(f * NC + k) * plane + p] = lb[f][k];
}

// The transposes of the Runge-Kutta combinations of Eq. (2Dfully-hweno), value by value, one pass
// each (every array has n values):
//   k_rk_seed:  muM = c1 x, muL = c2 x                       (the last stage's seeds from lam_in)
//   k_rk_mid:   lamB = c0 y + c1 x, muM = c2 x, muL = c3 x    (x = the last stage's VJP, y = lam_in)
//   k_rk_first: muM = x + y, muL = c3 x                       (x = the middle stage's VJP, y = lamB)
__global__ void k_rk_seed(long long n, double* __restrict__ muM, double* __restrict__ muL, double c1, double c2,
                          const double* __restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  muM[i] = c1 * v;
  muL[i] = c2 * v;
}
__global__ void k_rk_mid(long long n, double* __restrict__ lamB, double* __restrict__ muM, double* __restrict__ muL,
                         double c0, double c1, double c2, double c3, const double* __restrict__ x,
                         const double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  lamB[i] = fma(c0, y[i], c1 * v);
  muM[i] = c2 * v;
  muL[i] = c3 * v;
}
__global__ void k_rk_first(long long n, double* __restrict__ muM, double* __restrict__ muL, double c3,
                           const double* __restrict__ x, const double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  muM[i] = v + y[i];
  muL[i] = c3 * v;
}

}  // namespace hw

namespace hwh {
unsigned int bounds_take_adjoint(int* line) {
#ifdef HWENO_BOUNDS_CHECK
  return hw::bounds_take(line);
#else
  if (line) *line = 0;
  return 0;
#endif
}
}  // namespace hwh

namespace {

struct AdjLayout {
  size_t S1, S2, lam2, lam1, lamB, muM, muL, CU, CD, CM, total;
};

AdjLayout adj_layout(const hweno_ctx* h) {
  const size_t nst = hweno_state_doubles(h) * 8;
  const size_t nc = nc_of(h);
  const size_t nfx = (size_t)(h->nx + 1) * h->ny, nfy = h->dim == 2 ? (size_t)(h->ny + 1) * h->nx : 0;
  AdjLayout l;
  l.S1 = l.S2 = l.lam2 = l.lam1 = l.lamB = l.muM = l.muL = align_up(nst);
  l.CU = l.CD = align_up((nfx + nfy) * 4 * nc * 8);
  l.CM = align_up((size_t)h->dim * h->nx * h->ny * 5 * nc * 8);
  l.total = 7 * l.S1 + l.CU + l.CD + l.CM;
  return l;
}

struct AdjPtrs {
  double *S1, *S2, *lam2, *lam1, *lamB, *muM, *muL;
  hw::AdjWork aw;
};

AdjPtrs adj_ptrs(const hweno_ctx* h, void* ws) {
  const AdjLayout l = adj_layout(h);
  unsigned char* p = static_cast<unsigned char*>(ws);
  AdjPtrs a;
  double** arr[7] = {&a.S1, &a.S2, &a.lam2, &a.lam1, &a.lamB, &a.muM, &a.muL};
  for (int k = 0; k < 7; ++k) {
    *arr[k] = reinterpret_cast<double*>(p);
    p += l.S1;
  }
  a.aw.CU = reinterpret_cast<double*>(p);
  p += l.CU;
  a.aw.CD = reinterpret_cast<double*>(p);
  p += l.CD;
  a.aw.CM = reinterpret_cast<double*>(p);
  a.aw.scal = h->w.scal;
  return a;
}

template <int DIM>
int stage_vjp(const hweno_ctx* h, const Grid& g, const double* S, const double* alpha2, const double* muM,
              const double* muL, const hw::AdjWork& aw, double* lam) {
  const cudaStream_t st = h->stream;
  const unsigned bc = blocks_for(g.plane);
  // shared memory for the saved forward intermediates: one slot per thread and value
  constexpr int NC = DIM == 1 ? 3 : 4;
  constexpr size_t cell_sm = (size_t)hw::kCellSaved * NC * hw::kThreads * sizeof(double);
  constexpr size_t face_sm = (size_t)hw::kFaceSaved * NC * hw::kThreads * sizeof(double);
  if (cudaFuncSetAttribute(hw::k_adj_face<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)face_sm) !=
          cudaSuccess ||
      cudaFuncSetAttribute(hw::k_adj_cell<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_sm) !=
          cudaSuccess)
    return HWENO_ECUDA;
  hw::k_adj_cell<DIM><<<dim3(bc, DIM), hw::kThreads, cell_sm, st>>>(g, S, muM, aw);
  const long long nfx = (long long)(g.nx + 1) * g.ny;
  const long long nfy = DIM == 2 ? (long long)(g.ny + 1) * g.nx : 0;
  hw::k_adj_face<DIM><<<dim3(blocks_for(nfx > nfy ? nfx : nfy), DIM), hw::kThreads, face_sm, st>>>(g, S, muL, aw,
                                                                                                  alpha2);
  hw::k_adj_gather<DIM><<<bc, hw::kThreads, 0, st>>>(g, S, muM, muL, aw, lam);
  return cudaGetLastError() == cudaSuccess ? HWENO_OK : HWENO_ECUDA;
}

unsigned rk_blocks(const hweno_ctx* h) { return (unsigned)((hweno_state_doubles(h) + 255) / 256); }
long long rk_n(const hweno_ctx* h) { return (long long)hweno_state_doubles(h); }
int launch_status() { return cudaGetLastError() == cudaSuccess ? HWENO_OK : HWENO_ECUDA; }

}  // namespace

extern "C" size_t hweno_adjoint_workspace_bytes(const hweno_t* h) { return h ? adj_layout(h).total : 0; }

namespace {

// the three stage VJPs of one step, given the stage inputs S^n, S1, S2
int adjoint_from_stages(hweno_t* h, const AdjPtrs& a, const double* Sn, const double* S1, const double* S2, double dt,
                        const double* alpha6, const double* lam_in, double* lam_out) {
  const Grid g = grid_of(h);
  int rc;
  auto vjp = [&](const double* S, int st, const double* muM, const double* muL, double* lam) {
    return h->dim == 1 ? stage_vjp<1>(h, g, S, alpha6 + 2 * st, muM, muL, a.aw, lam)
                       : stage_vjp<2>(h, g, S, alpha6 + 2 * st, muM, muL, a.aw, lam);
  };
  // S^{n+1} = 1/3 B + 2/3 (M(S2) + dt L(S2)):  muM = 2/3 lam_in, muL = 2/3 dt lam_in
  hw::k_rk_seed<<<rk_blocks(h), 256, 0, h->stream>>>(rk_n(h), a.muM, a.muL, 2.0 / 3.0, 2.0 / 3.0 * dt, lam_in);
  if ((rc = launch_status())) return rc;
  if ((rc = vjp(S2, 2, a.muM, a.muL, a.lam2))) return rc;
  // S2 = 3/4 B + 1/4 (M(S1) + dt L(S1)):  lamB = 1/3 lam_in + 3/4 lam2, muM = 1/4 lam2, muL = 1/4 dt lam2
  hw::k_rk_mid<<<rk_blocks(h), 256, 0, h->stream>>>(rk_n(h), a.lamB, a.muM, a.muL, 1.0 / 3.0, 0.75, 0.25, 0.25 * dt,
                                                    a.lam2, lam_in);
  if ((rc = launch_status())) return rc;
  if ((rc = vjp(S1, 1, a.muM, a.muL, a.lam1))) return rc;
  // S1 = M(S^n) + dt L(S^n), B = M(S^n):  muM = lam1 + lamB, muL = dt lam1
  hw::k_rk_first<<<rk_blocks(h), 256, 0, h->stream>>>(rk_n(h), a.muM, a.muL, dt, a.lam1, a.lamB);
  if ((rc = launch_status())) return rc;
  if ((rc = vjp(Sn, 0, a.muM, a.muL, lam_out))) return rc;
  h->launches += 9 + 3;
  return HWENO_OK;
}

}  // namespace

extern "C" {

int hweno_adjoint_step(hweno_t* h, const double* Sn, double dt, const double* alpha6, const double* lam_in,
                       double* lam_out, void* adj_ws) {
  if (!h || !Sn || !alpha6 || !lam_in || !lam_out || !adj_ws) return HWENO_EINVAL;
  if (h->system != HWENO_EULER || h->var != 0) return HWENO_EINVAL;
  if (!(dt > 0.0) || ((uintptr_t)adj_ws & 255)) return HWENO_EINVAL;
  if (!h->ws) return HWENO_ESTATE;
  const AdjPtrs a = adj_ptrs(h, adj_ws);
  const size_t bytes = hweno_state_doubles(h) * 8;
  // forward stages 1 and 2 from S^n with the recorded alphas (the forward workspace is scratch)
  if (cudaMemcpyAsync(a.S1, Sn, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) return HWENO_ECUDA;
  int rc = stage_replay(h, a.S1, 0, dt, alpha6);
  if (rc) return rc;
  if (cudaMemcpyAsync(a.S2, a.S1, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess) return HWENO_ECUDA;
  rc = stage_replay(h, a.S2, 1, dt, alpha6 + 2);
  if (rc) return rc;
  return adjoint_from_stages(h, a, Sn, a.S1, a.S2, dt, alpha6, lam_in, lam_out);
}

int hweno_adjoint_step_stages(hweno_t* h, const double* Sn, const double* S1, const double* S2, double dt,
                              const double* alpha6, const double* lam_in, double* lam_out, void* adj_ws) {
  if (!h || !Sn || !S1 || !S2 || !alpha6 || !lam_in || !lam_out || !adj_ws) return HWENO_EINVAL;
  if (h->system != HWENO_EULER || h->var != 0) return HWENO_EINVAL;
  if (!(dt > 0.0) || ((uintptr_t)adj_ws & 255)) return HWENO_EINVAL;
  return adjoint_from_stages(h, adj_ptrs(h, adj_ws), Sn, S1, S2, dt, alpha6, lam_in, lam_out);
}

int hweno_step_replay_stages(hweno_t* h, double dt, const double* alpha6, double* S1_out, double* S2_out) {
  if (!h || !alpha6 || !S1_out || !S2_out || !(dt > 0.0)) return HWENO_EINVAL;
  if (!h->ws || !h->state) return HWENO_ESTATE;
  const size_t bytes = hweno_state_doubles(h) * 8;
  for (int st = 0; st < 3; ++st) {
    int rc = stage(h, h->state, h->state, 0, st, dt, st, nullptr, nullptr, alpha6 + 2 * st);
    if (rc) return rc;
    if (st < 2 && cudaMemcpyAsync(st == 0 ? S1_out : S2_out, h->state, bytes, cudaMemcpyDeviceToDevice,
                                  h->stream) != cudaSuccess)
      return HWENO_ECUDA;
  }
  return HWENO_OK;
}

int hweno_step_stages(hweno_t* h, double dt, double* S1_out, double* S2_out) {
  if (!h || !S1_out || !S2_out || !std::isfinite(dt)) return HWENO_EINVAL;
  if (!h->ws || !h->state) return HWENO_ESTATE;
  if (((uintptr_t)S1_out & 15) || ((uintptr_t)S2_out & 15)) return HWENO_EINVAL;
  const size_t bytes = hweno_state_doubles(h) * 8;
  for (int st = 0; st < 3; ++st) {
    int rc = stage(h, h->state, h->state, 0, st, dt, st, nullptr, nullptr);
    if (rc) return rc;
    if (st < 2 && cudaMemcpyAsync(st == 0 ? S1_out : S2_out, h->state, bytes, cudaMemcpyDeviceToDevice,
                                  h->stream) != cudaSuccess)
      return HWENO_ECUDA;
  }
  return HWENO_OK;
}

int hweno_step_replay(hweno_t* h, double dt, const double* alpha6) {
  if (!h || !alpha6 || !(dt > 0.0)) return HWENO_EINVAL;
  if (!h->ws || !h->state) return HWENO_ESTATE;
  for (int st = 0; st < 3; ++st) {
    int rc = stage(h, h->state, h->state, 0, st, dt, st, nullptr, nullptr, alpha6 + 2 * st);
    if (rc) return rc;
  }
  return HWENO_OK;
}

int hweno_step_record(hweno_t* h, double* rec7) {
  if (!h || !rec7) return HWENO_EINVAL;
  if (!h->ws) return HWENO_ESTATE;
  // dt of the last step, then the wavespeed slots of its three stages (bit patterns of doubles)
  if (cudaMemcpyAsync(rec7, h->w.scal, sizeof(double), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(rec7 + 1, h->w.alpha, 6 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  return HWENO_OK;
}

int hweno_stage_vjp(hweno_t* h, const double* S, const double* alpha2, const double* muM, const double* muL,
                    double* lam, void* adj_ws) {
  if (!h || !S || !alpha2 || !muM || !muL || !lam || !adj_ws) return HWENO_EINVAL;
  if (h->system != HWENO_EULER || h->var != 0) return HWENO_EINVAL;
  if ((uintptr_t)adj_ws & 255) return HWENO_EINVAL;
  const AdjPtrs a = adj_ptrs(h, adj_ws);
  const Grid g = grid_of(h);
  h->launches += 3;
  return h->dim == 1 ? stage_vjp<1>(h, g, S, alpha2, muM, muL, a.aw, lam)
                     : stage_vjp<2>(h, g, S, alpha2, muM, muL, a.aw, lam);
}

}  // extern "C"
