// Stage kernels of the HWENO-I scheme (Xie, Tao, Jiao, Zhang, arXiv 2411.11229) for sm_103a.
//
// One Runge-Kutta stage is three launches over the grid:
//   k_cell   per cell : wavespeed (LF alpha of the stage input), nodal fluxes f, h = f'(u) v (and
//                       the mixed-flux nodal values in 2D) for the D-terms (Eqs. Cd-1, DfDh, mixed),
//                       Euler primitives for the Roe averages, and the modified derivative v~
//                       (Eq. limiter) in the local characteristic fields of the cell.
//   k_face   per face : characteristic projection with the Roe-averaged eigenvectors, the HWENO
//                       interpolation of u and v to both sides of the face (Eqs. Pxi, P'xi, GHYZ,
//                       nonlinear, interp), back projection, and the numerical fluxes
//                       (Eqs. flux-1d, flux-LF, DfDh, mixed).
//   k_update per cell : conservative differences (Eqs. odeH / ode2H) and the SSP-RK3 combination
//                       with the modified derivative in the base (Eqs. fully-hweno, 2Dfully-hweno),
//                       in place; or L and M written out (rhs mode).
// The path is bound by the FP64 pipe (a few thousand FP64 operations per cell and stage against
// roughly a kilobyte of traffic), so the split keeps every warp's lanes busy on one kind of work
// and exchanges intermediates through L2/HBM, which has bandwidth to spare.
//
// VAR selects the scheme: 0 is the scheme of the paper with one boundary type on every side;
// 1 adds the runtime options (per-side boundary types with fixed-state sides, v^+/- with the
// nonlinear weights, the D-terms of Eq. Cd-2, the gravity source of Eq. euler2d-s); 2 is 1 with
// the per-cell characteristic decomposition (R2): k_cell interpolates both faces of every cell in
// the cell's own characteristic fields and k_face only forms the fluxes; k_r2_ghost supplies the
// face states of the ghost cells at the ends of every line.
#pragma once
#include "hweno_math.cuh"

namespace hw {

// Device views into the caller's workspace.
struct Work {
  double* B;     // stage base M(S^n): [NF][NC][plane]
  double* MD;    // modified derivatives (V~, W~): [DIM][NC][plane]
  double* NOD;   // nodal values per direction, normal frame: [DIM][NG][NC][plane]
  double* PRIM;  // Euler primitives (sqrt(rho), u[, v], H): [NP][plane]
  double* FX;    // x-face fluxes, original frame: [NF][NC][ny][nx+1]
  double* FY;    // y-face fluxes: [NF][NC][ny+1][nx]
  unsigned long long* alpha;  // wavespeed slots (bit patterns of non-negative doubles): slot s of
                              // direction d at alpha[s * astride + d]
  double* scal;               // [0] dt of the current step, [1] t, [2] t_end, [3] steps taken,
                              // [4..7] zero (read by fu_of; never written after creation)
  unsigned int* status;       // bit 0: non-physical state met
  long long astride;          // distance between slots (2 for a single grid)
  // R2 only: face states of every cell, normal frame:
  // FS [DIM][4][NC][plane] = (u^- and v^- at the right face, u^+ and v^+ at the left face);
  // GFS [DIM][2 ends][2][NC][gstride] = the low ghost's right-face and the high ghost's
  // left-face states of every line.
  double* FS;
  double* GFS;
  long long gstride;
  // local LF coefficients only: the spectral radius of every cell per direction [DIM][plane]
  double* WS;
};

constexpr int kThreads = 128;

// The units of FU in thread registers: a zero read at a per-thread address of the zeroed slots
// scal[4..7], so that the compiler can neither fold it nor keep it in a uniform register.
__device__ __forceinline__ FU fu_of(const double* scal) {
  const double z = scal[4 + (threadIdx.x & 3)];
  return FU{1.0 + z, -z, __double2hiint(z)};
}

template <int NC>
__device__ __forceinline__ void swap_frame(double* q) {
  if (NC == 4) {
    const double t = q[1];
    q[1] = q[2];
    q[2] = t;
  }
}

// max over the block of (a, b), then one atomicMax per block on the bit patterns
__device__ __forceinline__ void block_max2(double a, double b, unsigned long long* dst) {
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane == 0) {
      atomicMax(dst, dbl_bits(a));
      atomicMax(dst + 1, dbl_bits(b));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Modified derivative of one cell in one direction (normal frame).  U3/D3: cells i-1, i, i+1
// (D = derivative along the sweep; only i-1 and i+1 enter).  e: eigenvectors of the cell.  The
// limiter needs the characteristic fields only through the differences of neighbouring cells, so
// the two conserved differences are projected (equal neighbours give exactly zero).
template <int NC, int SYS>
__device__ __forceinline__ void modified_derivative(const double (&U3)[3][NC], const double (&D3)[3][NC],
                                                    const Eig<NC>& e, int dir, const Grid& g, double* out,
                                                    const FU& f) {
  double dU[2][NC], Dq[2][NC], Zm[NC], Zp[NC];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < NC; ++k) dU[q][k] = f.sub(U3[q + 1][k], U3[q][k]);
  if (SYS == SYS_EULER) {
    e.project(dU[0], Dq[0], f);
    e.project(dU[1], Dq[1], f);
    e.project(D3[0], Zm, f);
    e.project(D3[2], Zp, f);
  } else {
    Dq[0][0] = dU[0][0];
    Dq[1][0] = dU[1][0];
    Zm[0] = D3[0][0];
    Zp[0] = D3[2][0];
  }
  double ht[NC];
  const StencilK k = stencil_k(g, dir, f);
#pragma unroll
  for (int s = 0; s < NC; ++s) ht[s] = f.mul(cell_field_d(Dq[0][s], Dq[1][s], Zm[s], Zp[s], k, f), k.ih);
  if (SYS == SYS_EULER) {
    e.back(ht, out, f);
  } else {
    out[0] = ht[0];
  }
}

// The ghost cell of a fixed-state side: the side's state (normal frame), zero derivatives.
template <int NC, int SYS>
__device__ __forceinline__ void load_fixed(const Grid& g, int side, int dir, double* U, double* D) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    U[k] = g.fixU[side][k];
    D[k] = 0.0;
  }
  if (SYS == SYS_EULER && dir == 1) swap_frame<NC>(U);
}

// The three cells i-1, i, i+1 of cell (i, j) along direction d, through the boundary map (normal
// frame, mirrored or fixed where the map says so).  U3[1] is taken from Uc (already loaded).
template <int DIM, int SYS, int VAR, int NC>
__device__ __forceinline__ void load_stencil3(const Grid& g, const double* __restrict__ S, int d, int i, int j,
                                              int a0, const double* Uc, double (&U3)[3][NC], double (&D3)[3][NC]) {
  const long long plane = g.plane;
  const int n = d == 0 ? g.nx : g.ny;
  const int fld = d == 0 ? 1 : 2;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    bool refl, fixed = false;
    const int ac = VAR ? bc_map_ext(a0 - 1 + q, n, g.side[2 * d], g.side[2 * d + 1], refl, fixed)
                       : bc_map(a0 - 1 + q, n, g.bc, refl);
    const long long pc = HW_IDX(d == 0 ? (long long)j * g.nx + ac : (long long)ac * g.nx + i, plane);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      U3[q][k] = (q == 1 && Uc) ? Uc[k] : S[k * plane + pc];
      D3[q][k] = S[(fld * NC + k) * plane + pc];
    }
    if (SYS == SYS_EULER && d == 1) {
      swap_frame<NC>(U3[q]);
      swap_frame<NC>(D3[q]);
    }
    if (SYS == SYS_EULER) {
      mirror_U<NC>(U3[q], refl);
      mirror_D<NC>(D3[q], refl);
    }
    if (VAR && fixed) load_fixed<NC, SYS>(g, 2 * d + (a0 - 1 + q < 0 ? 0 : 1), d, U3[q], D3[q]);
  }
}

// R2: the modified derivative and the face states of one cell in one direction from its own
// stencil in its own characteristic fields (normal frame, derivatives unscaled).  The face values
// are the cell's state plus back-projected corrections; without the weighted-derivative option the
// face derivatives are linear in the stencil and are formed in conserved variables.
template <int NC, int SYS, bool VW>
__device__ __forceinline__ void r2_cell_vw(const double (&U3)[3][NC], const double (&D3)[3][NC], const Eig<NC>& e,
                                           int dir, const Grid& g, double* md, double (&fs)[4][NC], const FU& f) {
  double dU[2][NC], Dq[2][NC], Zm[NC], Zp[NC];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < NC; ++k) dU[q][k] = f.sub(U3[q + 1][k], U3[q][k]);
  if (!VW) {
    // the Hermite derivative of Eq. (P'xi) at the two faces (linear in the stencil)
    const double k21 = g.uvd[dir][0], k3 = g.uvd[dir][1];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      fs[1][k] = fma(k21, dU[1][k], fma(-k3, dU[0][k], fma(0.0625, D3[0][k], -0.1875 * D3[2][k])));
      fs[3][k] = fma(k21, dU[0][k], fma(-k3, dU[1][k], fma(-0.1875, D3[0][k], 0.0625 * D3[2][k])));
    }
  }
  if (SYS == SYS_EULER) {
    e.project(dU[0], Dq[0], f);
    e.project(dU[1], Dq[1], f);
    e.project(D3[0], Zm, f);
    e.project(D3[2], Zp, f);
  } else {
    Dq[0][0] = dU[0][0];
    Dq[1][0] = dU[1][0];
    Zm[0] = D3[0][0];
    Zp[0] = D3[2][0];
  }
  const double bc = SYS == SYS_EULER ? 0.0 : U3[1][0];
  const StencilK k = stencil_k(g, dir, f);
  double cm[NC], chm[NC], cp[NC], chp[NC], ht[NC];
#pragma unroll
  for (int s = 0; s < NC; ++s) {
    cell_faces_field<VW>(Dq[0][s], Dq[1][s], Zm[s], Zp[s], bc, k, g, dir, cm[s], chm[s], cp[s], chp[s], ht[s], f);
    ht[s] = f.mul(ht[s], k.ih);
  }
  if (SYS == SYS_EULER) {
    e.back_add(cm, U3[1], fs[0], f);
    e.back_add(cp, U3[1], fs[2], f);
    e.back(ht, md, f);
  } else {
    fs[0][0] = cm[0];
    fs[2][0] = cp[0];
    md[0] = ht[0];
  }
  if (VW) {
    if (SYS == SYS_EULER) {
      e.back(chm, fs[1], f);
      e.back(chp, fs[3], f);
    } else {
      fs[1][0] = chm[0];
      fs[3][0] = chp[0];
    }
  }
}

// r2_cell_vw with the weighted-derivative option read from the grid's flags (one code path each)
template <int NC, int SYS>
__device__ __forceinline__ void r2_cell(const double (&U3)[3][NC], const double (&D3)[3][NC], const Eig<NC>& e,
                                        int dir, const Grid& g, double* md, double (&fs)[4][NC], const FU& f) {
  if (g.flags & FLAG_V_WEIGHTED)
    r2_cell_vw<NC, SYS, true>(U3, D3, e, dir, g, md, fs, f);
  else
    r2_cell_vw<NC, SYS, false>(U3, D3, e, dir, g, md, fs, f);
}

// Cell work of one stage at cell p: primitives and wavespeeds (returned in wsx, wsy), nodal
// values per direction, modified derivatives (and, for R2, the face states of the cell).
template <int DIM, int SYS, int VAR = 0>
__device__ __forceinline__ void cell_body(const Grid& g, const double* __restrict__ S, const Work& w, long long p_in,
                                          double& wsx, double& wsy) {
  using T = Traits<DIM, SYS>;
  constexpr int NC = T::NC, NG = T::NG;
  const long long plane = g.plane;
  const long long p = HW_IDX(p_in, plane);
  const FU f = fu_of(w.scal);
  {
    const int i = (int)(p % g.nx), j = (int)(p / g.nx);
    double U[NC], V[NC], Wd[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      U[k] = S[k * plane + p];
      V[k] = S[(NC + k) * plane + p];
      if (DIM == 2) Wd[k] = S[(2 * NC + k) * plane + p];
    }
    // primitives and wavespeeds
    double u = 0, v = 0, pr = 0, ir = 0, H = 0, c = 0, ic = 0;
    if (SYS == SYS_EULER) {
      ir = rcp(U[0], f);
      u = f.mul(U[1], ir);
      if (DIM == 2) v = f.mul(U[2], ir);
      const double ke = DIM == 2 ? fma(U[1], u, f.mul(U[2], v)) : f.mul(U[1], u);
      pr = g.gm1 * fma(-0.5, ke, U[NC - 1]);
      H = f.mul(f.add(U[NC - 1], pr), ir);
      const double c2 = f.mul(g.gamma * pr, ir);
      ic = rsqrt(c2);
      c = f.mul(c2, ic);
      wsx = fabs(u) + c;
      wsy = DIM == 2 ? fabs(v) + c : 0.0;
      if (!(U[0] > 0.0) || !(pr > 0.0) || !isfinite(wsx) || !isfinite(wsy)) atomicOr(w.status, 1u);
      w.PRIM[p] = sqrt(U[0]);
      w.PRIM[plane + p] = u;
      if (DIM == 2) {
        w.PRIM[2 * plane + p] = v;
        w.PRIM[3 * plane + p] = H;
      } else {
        w.PRIM[2 * plane + p] = H;
      }
    } else if (SYS == SYS_BURGERS) {
      wsx = fabs(U[0]);
      wsy = DIM == 2 ? wsx : 0.0;
      if (!isfinite(wsx)) atomicOr(w.status, 1u);
    } else {
      wsx = fabs(g.ax);
      wsy = DIM == 2 ? fabs(g.ay) : 0.0;
    }
    if (VAR && (g.flags & FLAG_ALPHA_LOCAL)) {
      w.WS[p] = wsx;
      if (DIM == 2) w.WS[plane + p] = wsy;
    }
    // primitive derivatives along V and W (2D Euler: shared by the Jacobians of both directions)
    double pdV[3] = {0.0, 0.0, 0.0}, pdW[3] = {0.0, 0.0, 0.0};
    if (SYS == SYS_EULER && DIM == 2) {
      Phys<2, SYS_EULER>::prim_deriv(U, u, v, ir, V, g.gm1, pdV[0], pdV[1], pdV[2], f);
      Phys<2, SYS_EULER>::prim_deriv(U, u, v, ir, Wd, g.gm1, pdW[0], pdW[1], pdW[2], f);
    }
    // nodal values per direction (normal frame)
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      double Un[NC], Dn[NC], On[NC], F[NC], Hn[NC], Mx[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        Un[k] = U[k];
        Dn[k] = d == 0 ? V[k] : Wd[k];
        On[k] = d == 0 ? Wd[k] : V[k];
      }
      const double a = d == 0 ? g.ax : g.ay;
      if (SYS == SYS_EULER) {
        if (d == 1) {
          swap_frame<NC>(Un);
          swap_frame<NC>(Dn);
          swap_frame<NC>(On);
        }
        const double un = d == 0 ? u : v;
        F[0] = Un[1];
        F[1] = fma(Un[1], un, pr);
        if (DIM == 2) F[2] = f.mul(Un[2], un);
        F[NC - 1] = f.mul(f.add(Un[NC - 1], pr), un);
        if (DIM == 2) {
          // own-direction field (V in x, W in y) and the other one, each with its normal-velocity
          // derivative (u' in x, v' in y)
          const double* po = d == 0 ? pdV : pdW;
          const double* pt = d == 0 ? pdW : pdV;
          const double hp = f.add(U[NC - 1], pr);
          Phys<2, SYS_EULER>::jvp_apply(Un, Dn, un, po[d], po[2], hp, Hn, f);
          Phys<2, SYS_EULER>::jvp_apply(Un, On, un, pt[d], pt[2], hp, Mx, f);
        } else {
          Phys<1, SYS_EULER>::jvp_prim(Un, un, pr, ir, Dn, Hn, g.gm1, f);
        }
      } else {
        Phys<DIM, SYS>::flux(Un, F, a, g.gm1);
        Phys<DIM, SYS>::jvp(Un, Dn, Hn, a, g.gm1);
        if (DIM == 2) Phys<DIM, SYS>::jvp(Un, On, Mx, a, g.gm1);
      }
      double* nod = w.NOD + (long long)d * NG * NC * plane;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        nod[k * plane + p] = F[k];
        nod[(NC + k) * plane + p] = Hn[k];
        if (DIM == 2) nod[(2 * NC + k) * plane + p] = Mx[k];
      }
    }
    // modified derivatives (Eq. limiter), one per direction
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int a0 = d == 0 ? i : j;
      double U3[3][NC], D3[3][NC];
      load_stencil3<DIM, SYS, VAR, NC>(g, S, d, i, j, a0, U, U3, D3);
      Eig<NC> e;
      if (SYS == SYS_EULER) e.setup(d == 0 ? u : v, d == 0 ? v : u, H, c, ic, g.gm1);
      double out[NC];
      if (VAR == 2) {
        double fs[4][NC];
        r2_cell<NC, SYS>(U3, D3, e, d, g, out, fs, f);
        double* FSd = w.FS + (long long)d * 4 * NC * plane;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < NC; ++k) FSd[(q * NC + k) * plane + p] = fs[q][k];
      } else {
        modified_derivative<NC, SYS>(U3, D3, e, d, g, out, f);
      }
      if (SYS == SYS_EULER && d == 1) swap_frame<NC>(out);
#pragma unroll
      for (int k = 0; k < NC; ++k) w.MD[((long long)d * NC + k) * plane + p] = out[k];
    }
  }
}

template <int DIM, int SYS, int VAR>
__global__ void __launch_bounds__(kThreads) k_cell(Grid g, const double* __restrict__ S, Work w, int slot) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  double wsx = 0.0, wsy = 0.0;
  if (p < g.plane) cell_body<DIM, SYS, VAR>(g, S, w, p, wsx, wsy);
  block_max2(wsx, wsy, w.alpha + slot * w.astride);
}

// R1 face states: the interface values and derivatives from both sides of face k+1/2, from the
// states Uq and derivatives Zq (normal frame) of the cells k-1..k+2, interpolated in the
// characteristic fields of e (the Roe average at the face; unused for a scalar law).  The
// interpolation needs the fields only through differences of neighbouring cells and the
// derivatives: the three conserved differences are projected and the centre states added back in
// conserved variables.  VW: the weighted-derivative option.
template <int NC, int SYS, bool VW>
__device__ __forceinline__ void r1_face_states(const double (&Uq)[4][NC], const double (&Zq)[4][NC],
                                               const Eig<NC>& e, const Grid& g, int dir, double* Um, double* Up,
                                               double* Dm, double* Dp, const FU& f) {
  double dU[3][NC];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int k = 0; k < NC; ++k) dU[q][k] = f.sub(Uq[q + 1][k], Uq[q][k]);
  if (!VW) {
    // the Hermite derivative of Eq. (P'xi) at the face from both sides (linear in the stencil,
    // formed first so that the differences and derivatives are not held through the fields)
    const double k21 = g.uvd[dir][0], k3 = g.uvd[dir][1];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Dm[k] = fma(k21, dU[1][k], fma(-k3, dU[0][k], fma(0.0625, Zq[0][k], -0.1875 * Zq[2][k])));
      Dp[k] = fma(k21, dU[1][k], fma(-k3, dU[2][k], fma(-0.1875, Zq[1][k], 0.0625 * Zq[3][k])));
    }
  }
  double Dq[3][NC], Yq[4][NC];
  if (SYS == SYS_EULER) {
#pragma unroll
    for (int q = 0; q < 3; ++q) e.project(dU[q], Dq[q], f);
#pragma unroll
    for (int q = 0; q < 4; ++q) e.project(Zq[q], Yq[q], f);
  } else {
#pragma unroll
    for (int q = 0; q < 3; ++q) Dq[q][0] = dU[q][0];
#pragma unroll
    for (int q = 0; q < 4; ++q) Yq[q][0] = Zq[q][0];
  }
  // HWENO interpolation in each characteristic field: u^- from the stencil of cell k, u^+ from the
  // stencil of cell k+1 (mirror image)
  const double bm = SYS == SYS_EULER ? 0.0 : Uq[1][0], bp = SYS == SYS_EULER ? 0.0 : Uq[2][0];
  double cm[NC], chm[NC], cp[NC], chp[NC];
  const StencilK k = stencil_k(g, dir, f);
#pragma unroll
  for (int s = 0; s < NC; ++s)
    face_field_d<VW>(Dq[0][s], Dq[1][s], Dq[2][s], Yq[0][s], Yq[1][s], Yq[2][s], Yq[3][s], bm, bp, k, g, dir, cm[s],
                     chm[s], cp[s], chp[s], f);
  // back to conserved variables
  if (SYS == SYS_EULER) {
    e.back_add(cm, Uq[1], Um, f);
    e.back_add(cp, Uq[2], Up, f);
  } else {
    Um[0] = cm[0];
    Up[0] = cp[0];
  }
  if (VW) {
    if (SYS == SYS_EULER) {
      e.back(chm, Dm, f);
      e.back(chp, Dp, f);
    } else {
      Dm[0] = chm[0];
      Dp[0] = chp[0];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Face work of one stage: face f of direction dir (x faces: f = j (nx+1) + i; y faces:
// f = j nx + i), alpha = the LF coefficient of that direction.
template <int DIM, int SYS, int VAR = 0>
__device__ __forceinline__ void face_body(const Grid& g, const double* __restrict__ S, const Work& w, int dir,
                                          long long f, double alpha) {
  using T = Traits<DIM, SYS>;
  constexpr int NC = T::NC, NG = T::NG;
  const long long plane = g.plane;
  const FU fu = fu_of(w.scal);
  const int n = dir == 0 ? g.nx : g.ny;
  int fa, line;
  if (dir == 0) {
    line = (int)(f / (n + 1));
    fa = (int)(f % (n + 1));
  } else {
    fa = (int)(f / g.nx);
    line = (int)(f % g.nx);
  }
  // cells fa-2 .. fa+1 around face fa (between cells fa-1 and fa)
  long long pc[4];
  bool refl[4], fixed[4];
  int fside[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    fixed[q] = false;
    fside[q] = 2 * dir + (fa - 2 + q < 0 ? 0 : 1);
    const int a = VAR ? bc_map_ext(fa - 2 + q, n, g.side[2 * dir], g.side[2 * dir + 1], refl[q], fixed[q])
                      : bc_map(fa - 2 + q, n, g.bc, refl[q]);
    pc[q] = HW_IDX(dir == 0 ? (long long)line * g.nx + a : (long long)a * g.nx + line, plane);
  }
  const int fown = dir == 0 ? 1 : 2, foth = dir == 0 ? 2 : 1;
  double Um[NC], Up[NC], Dm[NC], Dp[NC];
  if (VAR == 2) {
    // R2: the face states were formed per cell (the low and high ghosts by k_r2_ghost)
    const double* FSd = w.FS + (long long)dir * 4 * NC * plane;
    const long long gs = w.gstride;
    const double* Glo = w.GFS + (long long)(dir * 2 + 0) * 2 * NC * gs;
    const double* Ghi = w.GFS + (long long)(dir * 2 + 1) * 2 * NC * gs;
    const long long gl = HW_IDX(line, gs);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      Um[k] = fa >= 1 ? FSd[(0 * NC + k) * plane + pc[1]] : Glo[(0 * NC + k) * gs + gl];
      Dm[k] = fa >= 1 ? FSd[(1 * NC + k) * plane + pc[1]] : Glo[(1 * NC + k) * gs + gl];
      Up[k] = fa < n ? FSd[(2 * NC + k) * plane + pc[2]] : Ghi[(0 * NC + k) * gs + gl];
      Dp[k] = fa < n ? FSd[(3 * NC + k) * plane + pc[2]] : Ghi[(1 * NC + k) * gs + gl];
    }
  } else {
    double Uq[4][NC], Zq[4][NC];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        Uq[q][k] = S[k * plane + pc[q]];
        Zq[q][k] = S[(fown * NC + k) * plane + pc[q]];
      }
      if (SYS == SYS_EULER && dir == 1) {
        swap_frame<NC>(Uq[q]);
        swap_frame<NC>(Zq[q]);
      }
      if (SYS == SYS_EULER) {
        mirror_U<NC>(Uq[q], refl[q]);
        mirror_D<NC>(Zq[q], refl[q]);
      }
      if (VAR && fixed[q]) load_fixed<NC, SYS>(g, fside[q], dir, Uq[q], Zq[q]);
    }
    // characteristic fields at the face: Roe average of the two adjacent cells
    Eig<NC> e;
    if (SYS == SYS_EULER) {
      const int ou = dir == 0 ? 1 : 2, ov = dir == 0 ? 2 : 1;
      const int oh = DIM == 2 ? 3 : 2;
      double sl = w.PRIM[pc[1]], sr = w.PRIM[pc[2]];
      // a mirrored neighbour has the opposite normal velocity
      double ul = neg_if(w.PRIM[ou * plane + pc[1]], refl[1]);
      double ur = neg_if(w.PRIM[ou * plane + pc[2]], refl[2]);
      double vl = 0, vr = 0;
      if (DIM == 2) {
        vl = w.PRIM[ov * plane + pc[1]];
        vr = w.PRIM[ov * plane + pc[2]];
      }
      double Hl = w.PRIM[oh * plane + pc[1]], Hr = w.PRIM[oh * plane + pc[2]];
      if (VAR && fixed[1]) {
        const double* P = g.fixP[fside[1]];
        sl = P[0];
        ul = P[ou];
        if (DIM == 2) vl = P[ov];
        Hl = P[oh];
      }
      if (VAR && fixed[2]) {
        const double* P = g.fixP[fside[2]];
        sr = P[0];
        ur = P[ou];
        if (DIM == 2) vr = P[ov];
        Hr = P[oh];
      }
      const double iw = rcp(fu.add(sl, sr), fu);
      const double ub = fu.mul(fma(sl, ul, fu.mul(sr, ur)), iw);
      const double vb = DIM == 2 ? fu.mul(fma(sl, vl, fu.mul(sr, vr)), iw) : 0.0;
      const double Hb = fu.mul(fma(sl, Hl, fu.mul(sr, Hr)), iw);
      const double c2 = g.gm1 * fma(-0.5, DIM == 2 ? fma(ub, ub, fu.mul(vb, vb)) : fu.mul(ub, ub), Hb);
      const double ic = rsqrt(c2);
      e.setup(ub, vb, Hb, fu.mul(c2, ic), ic, g.gm1);
    }
    if (VAR && (g.flags & FLAG_V_WEIGHTED))
      r1_face_states<NC, SYS, true>(Uq, Zq, e, g, dir, Um, Up, Dm, Dp, fu);
    else
      r1_face_states<NC, SYS, false>(Uq, Zq, e, g, dir, Um, Up, Dm, Dp, fu);
  }
  // local LF: the larger spectral radius of the two cells of the face
  if (VAR && (g.flags & FLAG_ALPHA_LOCAL)) {
    const double al = fixed[1] ? g.fixA[fside[1]] : w.WS[dir * plane + pc[1]];
    const double ar = fixed[2] ? g.fixA[fside[2]] : w.WS[dir * plane + pc[2]];
    alpha = fmax(al, ar);
  }
  // Lax-Friedrichs fluxes at the interpolated states (Eq. flux-LF)
  const double a_adv = dir == 0 ? g.ax : g.ay;
  double FUm[NC], FUp[NC], HDm[NC], HDp[NC];
  Phys<DIM, SYS>::flux_jvp(Um, Dm, FUm, HDm, a_adv, g.gm1, fu);
  Phys<DIM, SYS>::flux_jvp(Up, Dp, FUp, HDp, a_adv, g.gm1, fu);
  const double* nod = w.NOD + (long long)dir * NG * NC * plane;
  double* out = dir == 0 ? w.FX : w.FY;
  const long long oplane = dir == 0 ? (long long)g.ny * (g.nx + 1) : (long long)(g.ny + 1) * g.nx;
  const long long fo = HW_IDX(dir == 0 ? (long long)line * (g.nx + 1) + fa : (long long)fa * g.nx + line, oplane);
  const bool cd2 = VAR && (g.flags & FLAG_CD2) != 0;
  double fh[NC], hh[NC], mh[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    // nodal values of mirrored neighbours (normal frame): f and the mixed value change sign except
    // for the normal momentum, the normal-derivative flux changes sign only for the normal momentum
    const bool nm = k == 1;
    const bool s0 = refl[0] && !nm, s1 = refl[1] && !nm, s2 = refl[2] && !nm, s3 = refl[3] && !nm;
    double f0 = neg_if(nod[k * plane + pc[0]], s0), f1 = neg_if(nod[k * plane + pc[1]], s1);
    double f2 = neg_if(nod[k * plane + pc[2]], s2), f3 = neg_if(nod[k * plane + pc[3]], s3);
    // h at the outer nodes (Eq. Cd-1) or, for Cd-2, at the inner ones
    double ha = neg_if(nod[(NC + k) * plane + pc[cd2 ? 1 : 0]], refl[cd2 ? 1 : 0] && nm);
    double hb = neg_if(nod[(NC + k) * plane + pc[cd2 ? 2 : 3]], refl[cd2 ? 2 : 3] && nm);
    if (VAR) {
      // a fixed-state ghost: the side's flux, zero derivative fluxes
      if (fixed[0]) f0 = g.fixF[fside[0]][k];
      if (fixed[1]) f1 = g.fixF[fside[1]][k];
      if (fixed[2]) f2 = g.fixF[fside[2]][k];
      if (fixed[3]) f3 = g.fixF[fside[3]][k];
      if (fixed[cd2 ? 1 : 0]) ha = 0.0;
      if (fixed[cd2 ? 2 : 3]) hb = 0.0;
    }
    double Df, Dh;
    if (cd2) {
      // D-terms (Eqs. Cd-2, DfDh)
      Df = fma(DCoef2::cf, fu.add(fu.sub(f0, f1), fu.sub(f3, f2)), g.c2h[dir] * fu.sub(ha, hb));
      Dh = fma(g.e2fih[dir], fu.sub(f0, f3), fma(g.e2gih[dir], fu.sub(f1, f2), DCoef2::eh * fu.add(ha, hb)));
    } else {
      // D-terms (Eqs. Cd-1, DfDh)
      Df = fma(DCoef::cf, fu.add(fu.sub(f0, f1), fu.sub(f3, f2)), g.chh[dir] * fu.sub(ha, hb));
      Dh = fma(g.efih[dir], fu.sub(f0, f3), fma(g.egih[dir], fu.sub(f2, f1), DCoef::eh * fu.add(ha, hb)));
    }
    fh[k] = fma(0.5, fma(-alpha, fu.sub(Up[k], Um[k]), fu.add(FUm[k], FUp[k])), Df);
    hh[k] = fma(0.5, fma(-alpha, fu.sub(Dp[k], Dm[k]), fu.add(HDm[k], HDp[k])), Dh);
    if (DIM == 2) {
      double o0 = neg_if(nod[(2 * NC + k) * plane + pc[0]], s0);
      double o1 = neg_if(nod[(2 * NC + k) * plane + pc[1]], s1);
      double o2 = neg_if(nod[(2 * NC + k) * plane + pc[2]], s2);
      double o3 = neg_if(nod[(2 * NC + k) * plane + pc[3]], s3);
      if (VAR) {
        if (fixed[0]) o0 = 0.0;
        if (fixed[1]) o1 = 0.0;
        if (fixed[2]) o2 = 0.0;
        if (fixed[3]) o3 = 0.0;
      }
      // Eq. (mixed)
      mh[k] = fma(7.0 / 12.0, fu.add(o1, o2), (-1.0 / 12.0) * fu.add(o0, o3));
    }
  }
  if (SYS == SYS_EULER && dir == 1) {
    swap_frame<NC>(fh);
    swap_frame<NC>(hh);
    swap_frame<NC>(mh);
  }
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    out[k * oplane + fo] = fh[k];
    out[(fown * NC + k) * oplane + fo] = hh[k];
    if (DIM == 2) out[(foth * NC + k) * oplane + fo] = mh[k];
  }
}

// 2D: three blocks of 128 per SM, so that the stencil constants of the direction (StencilK) stay in
// registers; 1D: four
template <int DIM, int SYS, int VAR>
__global__ void __launch_bounds__(kThreads, DIM == 2 ? 3 : 4) k_face(Grid g, const double* __restrict__ S, Work w,
                                                                    int slot) {
  const int dir = blockIdx.y;
  const int n = dir == 0 ? g.nx : g.ny;
  const int nlines = dir == 0 ? g.ny : g.nx;
  const long long f = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (f >= (long long)(n + 1) * nlines) return;
  face_body<DIM, SYS, VAR>(g, S, w, dir, f, __longlong_as_double((long long)w.alpha[slot * w.astride + dir]));
}

// ---------------------------------------------------------------------------------------------
// Update of one cell p.  mode 0: Runge-Kutta stage in place, S = a B + b (M + dt L) (stage 0:
// B := M, S = M + dt L).  mode 1: write L and M to Lout, Mout.
template <int DIM, int SYS, int VAR = 0>
__device__ __forceinline__ void update_body(const Grid& g, double* __restrict__ S, const Work& w, int mode, int stage,
                                            double a_k, double b_k, double dt, long long p_in,
                                            double* __restrict__ Lout, double* __restrict__ Mout) {
  using T = Traits<DIM, SYS>;
  constexpr int NC = T::NC, NF = T::NF;
  constexpr bool SRC = VAR != 0 && DIM == 2 && SYS == SYS_EULER;  // gravity source possible
  const long long plane = g.plane;
  const long long p = HW_IDX(p_in, plane);
  const int i = (int)(p % g.nx), j = (int)(p / g.nx);
  const long long oplx = (long long)g.ny * (g.nx + 1), oply = (long long)(g.ny + 1) * g.nx;
  const long long px = HW_IDX((long long)j * (g.nx + 1) + i, oplx - 1);  // faces px and px + 1
  // the stage's constants copied into thread registers (exactly: c 1 + (-0) = c), so that every
  // FP64 instruction below has register operands (see FU)
  const FU fu = fu_of(w.scal);
  const double mix = fu.reg(-g.inv_dx), miy = fu.reg(-g.inv_dy);
  const double akr = fu.reg(a_k), bkr = fu.reg(b_k);
  // the Runge-Kutta stage b (M + dt L) with dt L = (dt mix) dF + (dt miy) dG (+ dt source): the
  // coefficients of the two flux differences taken as one product each, b dt (-1/h) (b = 1 at the
  // first stage)
  const double bdt = fu.mul(bkr, fu.reg(dt));
  const double cx = fu.mul(bdt, mix), cy = fu.mul(bdt, miy);
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    // Eq. (euler2d-s): field f gains g (0, 0, S_f[rho], S_f[rho nu]) (read before S is overwritten)
    double src2 = 0.0, src3 = 0.0;
    if (SRC && g.grav != 0.0) {
      src2 = g.grav * S[(f * NC + 0) * plane + p];
      src3 = g.grav * S[(f * NC + 2) * plane + p];
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const int fk = f * NC + k;
      const double dF = fu.sub(w.FX[fk * oplx + px + 1], w.FX[fk * oplx + px]);
      const double dG = DIM == 2 ? fu.sub(w.FY[fk * oply + p + g.nx], w.FY[fk * oply + p]) : 0.0;
      const double M = f == 0 ? S[fk * plane + p] : w.MD[((long long)(f - 1) * NC + k) * plane + p];
      if (mode == 1) {
        // L = -(F_{i+1/2} - F_{i-1/2}) / dx [- (G_{j+1/2} - G_{j-1/2}) / dy] [+ source]
        double L = fu.mul(dF, mix);
        if (DIM == 2) L = fma(dG, miy, L);
        if (SRC && k == 2) L = fu.add(L, src2);
        if (SRC && k == 3) L = fu.add(L, src3);
        Lout[fk * plane + p] = L;
        Mout[fk * plane + p] = M;
        continue;
      }
      // b M + b dt L
      double v = stage == 0 ? M : fu.mul(bkr, M);
      if (SRC && k == 2) v = fma(bdt, src2, v);
      if (SRC && k == 3) v = fma(bdt, src3, v);
      if (DIM == 2) v = fma(cy, dG, v);
      v = fma(cx, dF, v);
      if (stage == 0) {
        w.B[fk * plane + p] = M;
        S[fk * plane + p] = v;
      } else {
        S[fk * plane + p] = fma(akr, w.B[fk * plane + p], v);
      }
    }
  }
}

// The step size of a stage: dt_fixed > 0, or (dt_fixed <= 0) at stage 0 the CFL step from the
// wavespeed slot (clamped to t_end); stages 1 and 2 reuse the value stored in scal[0].
template <int DIM>
__device__ __forceinline__ double stage_dt(const Grid& g, const Work& w, int stage, double dt_fixed, int slot) {
  if (stage != 0) return w.scal[0];
  if (dt_fixed > 0.0) return dt_fixed;
  const double axs = __longlong_as_double((long long)w.alpha[slot * w.astride]);
  const double ays = __longlong_as_double((long long)w.alpha[slot * w.astride + 1]);
  double dt = DIM == 2 ? g.cfl / fma(axs, g.inv_dx, ays * g.inv_dy) : g.cfl * g.dx / axs;
  const double t = w.scal[1], te = w.scal[2];
  if (te > 0.0 && t + dt > te) dt = fmax(te - t, 0.0);
  return dt;
}

// dt of stage 0 is stored in scal[0] by block 0 and reused by stages 1 and 2; the time advances
// at stage 2.
template <int DIM, int SYS, int VAR>
__global__ void __launch_bounds__(kThreads) k_update(Grid g, double* __restrict__ S, Work w, int mode, int stage,
                                                      double a_k, double b_k, double dt_fixed, int slot,
                                                      double* __restrict__ Lout, double* __restrict__ Mout) {
  __shared__ double s_dt;
  if (mode == 0) {
    if (threadIdx.x == 0) {
      const double dt = stage_dt<DIM>(g, w, stage, dt_fixed, slot);
      if (stage == 0 && blockIdx.x == 0) w.scal[0] = dt;
      s_dt = dt;
    }
    __syncthreads();
  }
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= g.plane) return;
  const double dt = mode == 0 ? s_dt : 0.0;
  // a CFL step at the end time has dt = 0: it leaves the state as it is, so that steps issued
  // past the end time (without waiting for the host) change nothing
  if (mode == 0 && dt_fixed <= 0.0 && dt == 0.0) return;
  update_body<DIM, SYS, VAR>(g, S, w, mode, stage, a_k, b_k, dt, p, Lout, Mout);
  if (mode == 0 && stage == 2 && p == 0) {
    w.scal[1] += dt;
    w.scal[3] += 1.0;  // steps taken
  }
}

// R2: face states of the ghost cells at both ends of every line (the low ghost's right-face
// state, the high ghost's left-face state), from the ghost's own stencil and characteristic
// fields through the boundary map.  Threads: [dir][end][line], gstride lines per (dir, end).
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_r2_ghost(Grid g, const double* __restrict__ S, Work w) {
  constexpr int NC = Traits<DIM, SYS_EULER>::NC;
  const long long gs = w.gstride;
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  const int dir = (int)(t / (2 * gs));
  const int end = (int)((t / gs) % 2);
  const int line = (int)(t % gs);
  if (dir >= DIM) return;
  const int n = dir == 0 ? g.nx : g.ny, nlines = dir == 0 ? g.ny : g.nx;
  if (line >= nlines) return;
  const int a0 = end == 0 ? -1 : n;
  const int i = dir == 0 ? 0 : line, j = dir == 0 ? line : 0;  // the line's coordinates
  double U3[3][NC], D3[3][NC];
  load_stencil3<DIM, SYS_EULER, 1, NC>(g, S, dir, i, j, a0, nullptr, U3, D3);
  // eigenvectors of the ghost's own state (normal frame)
  const double* U = U3[1];
  const double ir = rcp(U[0]);
  const double u = U[1] * ir, v = DIM == 2 ? U[2] * ir : 0.0;
  const double ke = DIM == 2 ? fma(U[1], u, U[2] * v) : U[1] * u;
  const double pr = g.gm1 * fma(-0.5, ke, U[NC - 1]);
  const double H = (U[NC - 1] + pr) * ir;
  const double c2 = g.gamma * pr * ir;
  const double ic = rsqrt(c2);
  Eig<NC> e;
  e.setup(u, v, H, c2 * ic, ic, g.gm1);
  double md[NC], fs[4][NC];
  r2_cell<NC, SYS_EULER>(U3, D3, e, dir, g, md, fs, fu_of(w.scal));
  double* G = w.GFS + (long long)(dir * 2 + end) * 2 * NC * gs;
  const int q0 = end == 0 ? 0 : 2;
  const long long gl = HW_IDX(line, gs);
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    G[(0 * NC + k) * gs + gl] = fs[q0][k];
    G[(1 * NC + k) * gs + gl] = fs[q0 + 1][k];
  }
}

// alpha of a state only (hweno_max_wavespeed)
template <int DIM, int SYS>
__global__ void __launch_bounds__(kThreads) k_wavespeed(Grid g, const double* __restrict__ S, Work w, int slot) {
  constexpr int NC = Traits<DIM, SYS>::NC;
  const long long plane = g.plane;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  double wsx = 0.0, wsy = 0.0;
  if (p < plane) {
    if (SYS == SYS_EULER) {
      double U[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) U[k] = S[k * plane + p];
      const double ir = rcp(U[0]);
      const double u = U[1] * ir, v = DIM == 2 ? U[2] * ir : 0.0;
      const double ke = DIM == 2 ? fma(U[1], u, U[2] * v) : U[1] * u;
      const double pr = g.gm1 * fma(-0.5, ke, U[NC - 1]);
      const double c = sqrt(g.gamma * pr * ir);
      wsx = fabs(u) + c;
      wsy = DIM == 2 ? fabs(v) + c : 0.0;
      if (!(U[0] > 0.0) || !(pr > 0.0) || !isfinite(wsx) || !isfinite(wsy)) atomicOr(w.status, 1u);
    } else if (SYS == SYS_BURGERS) {
      wsx = fabs(S[p]);
      wsy = DIM == 2 ? wsx : 0.0;
    } else {
      wsx = fabs(g.ax);
      wsy = DIM == 2 ? fabs(g.ay) : 0.0;
    }
  }
  block_max2(wsx, wsy, w.alpha + slot * w.astride);
}

}  // namespace hw
