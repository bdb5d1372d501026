// Host-side internals shared by the translation units of libhweno.so (not part of the ABI):
// the handle, the workspace layout, the folded kernel constants and the launch helpers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hweno.h"
#include "hweno_kernels.cuh"


namespace hwh {

using hw::Grid;
using hw::Work;

struct Launchers {
  void (*cell)(const Grid&, const double*, const Work&, int, cudaStream_t);
  void (*face)(const Grid&, const double*, const Work&, int, cudaStream_t);
  void (*update)(const Grid&, double*, const Work&, int, int, double, double, double, int, double*, double*,
                 cudaStream_t);
  void (*wavespeed)(const Grid&, const double*, const Work&, int, cudaStream_t);
  void (*ghost)(const Grid&, const double*, const Work&, cudaStream_t);  // R2 only, else null
};

inline unsigned blocks_for(long long n) { return (unsigned)((n + hw::kThreads - 1) / hw::kThreads); }

template <int DIM, int SYS, int VAR>
struct L {
  static void cell(const Grid& g, const double* S, const Work& w, int slot, cudaStream_t st) {
    hw::k_cell<DIM, SYS, VAR><<<blocks_for(g.plane), hw::kThreads, 0, st>>>(g, S, w, slot);
  }
  static void face(const Grid& g, const double* S, const Work& w, int slot, cudaStream_t st) {
    const long long nfx = (long long)(g.nx + 1) * g.ny;
    const long long nfy = DIM == 2 ? (long long)(g.ny + 1) * g.nx : 0;
    dim3 grid(blocks_for(nfx > nfy ? nfx : nfy), DIM);
    hw::k_face<DIM, SYS, VAR><<<grid, hw::kThreads, 0, st>>>(g, S, w, slot);
  }
  static void update(const Grid& g, double* S, const Work& w, int mode, int stage, double a, double b,
                     double dt, int slot, double* Lo, double* Mo, cudaStream_t st) {
    hw::k_update<DIM, SYS, VAR><<<blocks_for(g.plane), hw::kThreads, 0, st>>>(g, S, w, mode, stage, a, b, dt, slot,
                                                                            Lo, Mo);
  }
  static void wavespeed(const Grid& g, const double* S, const Work& w, int slot, cudaStream_t st) {
    hw::k_wavespeed<DIM, SYS><<<blocks_for(g.plane), hw::kThreads, 0, st>>>(g, S, w, slot);
  }
  static void ghost(const Grid& g, const double* S, const Work& w, cudaStream_t st) {
    hw::k_r2_ghost<DIM><<<blocks_for(2LL * DIM * w.gstride), hw::kThreads, 0, st>>>(g, S, w);
  }
  static constexpr Launchers table() {
    return Launchers{&cell, &face, &update, &wavespeed, VAR == 2 ? &ghost : nullptr};
  }
};

// [VAR][dim - 1][system]; R2 exists for the Euler equations only (for a scalar law the per-cell
// and per-face bases coincide, and the host runs VAR 1)
static const Launchers kTable[3][2][3] = {
    {{L<1, hw::SYS_ADV, 0>::table(), L<1, hw::SYS_BURGERS, 0>::table(), L<1, hw::SYS_EULER, 0>::table()},
     {L<2, hw::SYS_ADV, 0>::table(), L<2, hw::SYS_BURGERS, 0>::table(), L<2, hw::SYS_EULER, 0>::table()}},
    {{L<1, hw::SYS_ADV, 1>::table(), L<1, hw::SYS_BURGERS, 1>::table(), L<1, hw::SYS_EULER, 1>::table()},
     {L<2, hw::SYS_ADV, 1>::table(), L<2, hw::SYS_BURGERS, 1>::table(), L<2, hw::SYS_EULER, 1>::table()}},
    {{L<1, hw::SYS_ADV, 1>::table(), L<1, hw::SYS_BURGERS, 1>::table(), L<1, hw::SYS_EULER, 2>::table()},
     {L<2, hw::SYS_ADV, 1>::table(), L<2, hw::SYS_BURGERS, 1>::table(), L<2, hw::SYS_EULER, 2>::table()}}};

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace hwh

struct hweno_ctx {
  int dim, system, bc;
  int64_t nx, ny;
  double dx, dy, gamma;
  double gamma0, d0, eps, cfl, ax, ay;
  // extended scheme (hweno_create_ex); var = 0 for the scheme of the paper with one boundary
  // type, 1 with any extension, 2 with the per-cell characteristic decomposition (Euler)
  int var, flags;
  int side[4];
  double grav;
  double fixed[4][4];
  cudaStream_t stream;
  double* state;
  unsigned char* ws;
  hw::Work w;
  long long launches;
  // optional per-kernel timing: events recorded around the three launches of every stage
  bool profiling;
  std::vector<cudaEvent_t> events;  // groups of 4: before cell, before face, before update, after
  double kernel_ms[3];
  long long kernel_n[3];
};

namespace hwh {

inline int nc_of(const hweno_ctx* h) { return h->system == HWENO_EULER ? (h->dim == 1 ? 3 : 4) : 1; }
inline int nf_of(const hweno_ctx* h) { return h->dim + 1; }
inline int ng_of(const hweno_ctx* h) { return h->dim == 2 ? 3 : 2; }
inline int np_of(const hweno_ctx* h) { return h->system == HWENO_EULER ? (h->dim == 2 ? 4 : 3) : 0; }

// workspace sub-buffers in bytes, in layout order
struct Layout {
  size_t B, MD, NOD, PRIM, FX, FY, alpha, scal, status, FS, GFS, WS, total;
};

inline long long gstride_of(const hweno_ctx* h) { return h->nx > h->ny ? h->nx : h->ny; }

inline Layout layout_of(const hweno_ctx* h) {
  const size_t plane = (size_t)h->nx * h->ny;
  const size_t nc = nc_of(h), nf = nf_of(h);
  Layout l;
  l.B = align_up(nf * nc * plane * 8);
  l.MD = align_up((size_t)h->dim * nc * plane * 8);
  l.NOD = align_up((size_t)h->dim * ng_of(h) * nc * plane * 8);
  l.PRIM = align_up((size_t)np_of(h) * plane * 8 + 8);
  l.FX = align_up(nf * nc * (size_t)h->ny * (h->nx + 1) * 8);
  l.FY = h->dim == 2 ? align_up(nf * nc * (size_t)(h->ny + 1) * h->nx * 8) : 0;
  l.alpha = align_up(8 * 8);
  l.scal = align_up(8 * 8);
  l.status = align_up(16);
  l.FS = h->var == 2 ? align_up((size_t)h->dim * 4 * nc * plane * 8) : 0;
  l.GFS = h->var == 2 ? align_up((size_t)h->dim * 4 * nc * (size_t)gstride_of(h) * 8) : 0;
  l.WS = (h->var != 0 && (h->flags & HWENO_FLAG_ALPHA_LOCAL)) ? align_up((size_t)h->dim * plane * 8) : 0;
  l.total = l.B + l.MD + l.NOD + l.PRIM + l.FX + l.FY + l.alpha + l.scal + l.status + l.FS + l.GFS + l.WS;
  return l;
}

inline Grid grid_of(const hweno_ctx* h) {
  Grid g;
  g.nx = (int)h->nx;
  g.ny = (int)h->ny;
  g.bc = h->bc;
  g.flags = h->flags;
  g.plane = (long long)h->nx * h->ny;
  g.dx = h->dx;
  g.dy = h->dy;
  g.inv_dx = 1.0 / h->dx;
  g.inv_dy = 1.0 / h->dy;
  g.gamma = h->gamma;
  g.gm1 = h->gamma - 1.0;
  g.ax = h->ax;
  g.ay = h->ay;
  g.g0 = h->gamma0;
  g.g1 = 0.5 * (1.0 - h->gamma0);
  g.d0 = h->d0;
  g.d1 = 0.5 * (1.0 - h->d0);
  g.eps = h->eps;
  g.cfl = h->cfl;
  // folded constants (see hw::Grid)
  const double g1 = g.g1;
  const double cr[5] = {(-0.125 + 0.5 * g1) / g1, (0.5625 - 2.0 * g1) / g1, (0.5625 - 0.5 * g1) / g1,
                        -0.046875 / g1, -0.140625 / g1};
  const double cl[5] = {(0.5625 - 0.5 * g1) / g1, (0.5625 - 2.0 * g1) / g1, (-0.125 + 0.5 * g1) / g1,
                        0.140625 / g1, 0.046875 / g1};
  for (int k = 0; k < 5; ++k) {
    g.cr[k] = cr[k];
    g.cl[k] = cl[k];
  }
  // the centre-value-free forms: right face on (d01, d12, hvm, hvp) of the stencil {i-1, i, i+1};
  // left face (mirror) on (d_{i,i+1} of its own stencil's first pair, second pair, h v_{i-1}, h v_{i+1})
  const double dm[4] = {-cr[0], cr[2], cr[3], cr[4]};
  const double dp[4] = {-cl[0], cl[2], cl[3], cl[4]};
  g.G = g.g0 / g1;
  g.cdu = (0.75 - g.d1) / g.d1;
  const double csv = 0.25 / g.d1;
  g.Gd = g.d0 / g.d1;
  // The smoothness indicator beta0 of Eq. (GHYZ) as two quadratic forms.  Its linear forms
  // (coefficients on (h sv, du) and on (h dv, d2)) with their weights:
  //   a1 + a3/4 = (-3/16, 11/16), weight 1;   a3 = (1/4, -1/4), weight 781/20;
  //   a2 + 63/130 a4 = (67/520, 197/260), weight 13/3;   a4 = (-1/4, -1/2), weight 1421461/2275.
  // Each pair makes s X^2 + 2 q X Y + r Y^2 = s (X + (q/s) Y)^2 + T Y^2 with T = det / s, det the
  // weighted square of the pair's 2x2 determinant.
  struct Pair {
    double s, q, T;
  };
  auto pair = [](const double* f, double wf, const double* k, double wk) {
    Pair o;
    o.s = wf * f[0] * f[0] + wk * k[0] * k[0];
    o.q = wf * f[0] * f[1] + wk * k[0] * k[1];
    const double m = f[0] * k[1] - f[1] * k[0];
    o.T = wf * wk * m * m / o.s;
    return o;
  };
  const double fA[2] = {-3.0 / 16.0, 11.0 / 16.0}, fC[2] = {0.25, -0.25};
  const double fB[2] = {67.0 / 520.0, 197.0 / 260.0}, fD[2] = {-0.25, -0.5};
  const Pair p1 = pair(fA, 1.0, fC, 781.0 / 20.0), p2 = pair(fB, 13.0 / 3.0, fD, 1421461.0 / 2275.0);
  g.bT1 = p1.T;
  g.bT2 = p2.T;
  const double hs[2] = {h->dx, h->dy};
  for (int d = 0; d < 2; ++d) {
    g.h[d] = hs[d];
    g.ih[d] = 1.0 / hs[d];
    g.chh[d] = hw::DCoef::ch * hs[d];
    g.efih[d] = hw::DCoef::ef / hs[d];
    g.egih[d] = hw::DCoef::eg / hs[d];
    g.hih[d] = 0.5 / hs[d];
    g.c2h[d] = hw::DCoef2::ch * hs[d];
    // unscaled-derivative constants (see hw::Grid)
    g.bS1[d] = p1.s * hs[d] * hs[d];
    g.bN1[d] = p1.q / (p1.s * hs[d]);
    g.bS2[d] = p2.s * hs[d] * hs[d];
    g.bN2[d] = p2.q / (p2.s * hs[d]);
    g.udm[d][0] = dm[0];
    g.udm[d][1] = dm[1];
    g.udm[d][2] = dm[2] * hs[d];
    g.udm[d][3] = dm[3] * hs[d];
    g.udp[d][0] = dp[0];
    g.udp[d][1] = dp[1];
    g.udp[d][2] = dp[2] * hs[d];
    g.udp[d][3] = dp[3] * hs[d];
    g.uvd[d][0] = 1.3125 / hs[d];
    g.uvd[d][1] = 0.1875 / hs[d];
    g.ucsv[d] = csv * hs[d];
    g.e2fih[d] = hw::DCoef2::ef / hs[d];
    g.e2gih[d] = hw::DCoef2::eg / hs[d];
  }
  g.ig1 = 1.0 / g1;
  g.grav = h->grav;
  for (int sd = 0; sd < 4; ++sd) {
    g.side[sd] = h->side[sd];
    g.fixA[sd] = 0.0;
    for (int k = 0; k < 4; ++k) g.fixU[sd][k] = g.fixP[sd][k] = g.fixF[sd][k] = 0.0;
    if (h->side[sd] != hw::BC_FIXED) continue;
    const double* U = h->fixed[sd];
    for (int k = 0; k < 4; ++k) g.fixU[sd][k] = U[k];
    const int nc = nc_of(h);
    if (h->system != HWENO_EULER) {
      // scalar: the flux of the state along the side's normal, and |f'(u)|
      const double a = sd < 2 ? h->ax : h->ay;
      g.fixF[sd][0] = h->system == HWENO_ADVECTION ? a * U[0] : 0.5 * U[0] * U[0];
      g.fixA[sd] = h->system == HWENO_ADVECTION ? std::fabs(a) : std::fabs(U[0]);
      continue;
    }
    // primitives in the original frame, flux in the side's normal frame
    const double rho = U[0], u = U[1] / rho, v = h->dim == 2 ? U[2] / rho : 0.0, E = U[nc - 1];
    const double p = (h->gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v));
    const double H = (E + p) / rho;
    g.fixP[sd][0] = std::sqrt(rho);
    g.fixP[sd][1] = u;
    if (h->dim == 2) {
      g.fixP[sd][2] = v;
      g.fixP[sd][3] = H;
    } else {
      g.fixP[sd][2] = H;
    }
    const double un = sd < 2 ? u : v, mn = rho * un, mt = sd < 2 ? U[2] : U[1];
    g.fixA[sd] = std::fabs(un) + std::sqrt(h->gamma * p / rho);
    g.fixF[sd][0] = mn;
    g.fixF[sd][1] = mn * un + p;
    if (h->dim == 2) {
      g.fixF[sd][2] = mt * un;
      g.fixF[sd][3] = (E + p) * un;
    } else {
      g.fixF[sd][2] = (E + p) * un;
    }
  }
  return g;
}

inline int cuda_status() { return cudaGetLastError() == cudaSuccess ? HWENO_OK : HWENO_ECUDA; }

inline int read_status(hweno_ctx* h) {
  unsigned int st = 0;
  if (cudaMemcpyAsync(&st, h->w.status, sizeof(st), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HWENO_ECUDA;
  return st ? HWENO_ENONPHYS : HWENO_OK;
}

inline const Launchers& launchers(const hweno_ctx* h) { return kTable[h->var][h->dim - 1][h->system]; }

// one spatial-operator evaluation: cell, face; then update in the requested mode
// alpha_override (device, 2 doubles, may be null): LF coefficients to use instead of the
// wavespeeds of S_in (the recorded alphas of an adjoint replay)
inline int stage(hweno_ctx* h, const double* S_in, double* S_out, int mode, int st, double dt, int slot, double* Lo,
          double* Mo, const double* alpha_override = nullptr) {
  const Grid g = grid_of(h);
  const Launchers& f = launchers(h);
  if (cudaMemsetAsync(h->w.alpha + 2 * slot, 0, 2 * sizeof(unsigned long long), h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  if (h->profiling) {
    for (int k = 0; k < 4; ++k)
      if (cudaEventCreate(&ev[k]) != cudaSuccess) return HWENO_ECUDA;
    for (int k = 0; k < 4; ++k) h->events.push_back(ev[k]);
  }
  static const double a_k[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double b_k[3] = {1.0, 0.25, 2.0 / 3.0};
  if (ev[0]) cudaEventRecord(ev[0], h->stream);
  f.cell(g, S_in, h->w, slot, h->stream);
  if (f.ghost) {
    f.ghost(g, S_in, h->w, h->stream);
    h->launches += 1;
  }
  if (alpha_override &&
      cudaMemcpyAsync(h->w.alpha + slot * h->w.astride, alpha_override, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                      h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  if (ev[1]) cudaEventRecord(ev[1], h->stream);
  // LF coefficients held for the whole step: stages 2 and 3 read the first stage's slot
  const bool held = h->var != 0 && (h->flags & HWENO_FLAG_ALPHA_STEP) && mode == 0 && st > 0;
  f.face(g, S_in, h->w, held ? slot - st : slot, h->stream);
  if (ev[2]) cudaEventRecord(ev[2], h->stream);
  f.update(g, S_out, h->w, mode, st, a_k[st], b_k[st], dt, slot, Lo, Mo, h->stream);
  if (ev[3]) cudaEventRecord(ev[3], h->stream);
  h->launches += 3;
  return cuda_status();
}

// one forward stage in place with fixed dt and the given LF coefficients
// bounds-checked build: the out-of-range index records of the batched and adjoint translation
// units (count since the last call, first source line; 0 in a normal build)
unsigned int bounds_take_batch(int* line);
unsigned int bounds_take_adjoint(int* line);

inline int stage_replay(hweno_ctx* h, double* S, int st, double dt, const double* alpha2_dev) {
  return stage(h, S, S, 0, st, dt, st, nullptr, nullptr, alpha2_dev);
}

}  // namespace hwh
