// C ABI of libhweno.so: see include/hweno.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <atomic>
#include <new>
#include <vector>

#include "../../include/hweno.h"
#include "hweno_kernels.cuh"

namespace hw {
// applies the library's FP64 reciprocal to n values (accuracy self-test)
__global__ void k_rcp_check(const double* __restrict__ x, double* __restrict__ r, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = rcp(x[i]);
}
}  // namespace hw

namespace {

using hw::Grid;
using hw::Work;

struct Launchers {
  void (*cell)(const Grid&, const double*, const Work&, int, cudaStream_t);
  void (*face)(const Grid&, const double*, const Work&, int, cudaStream_t);
  void (*update)(const Grid&, double*, const Work&, int, int, double, double, double, int, double*, double*,
                 cudaStream_t);
  void (*wavespeed)(const Grid&, const double*, const Work&, int, cudaStream_t);
};

inline unsigned blocks_for(long long n) { return (unsigned)((n + hw::kThreads - 1) / hw::kThreads); }

template <int DIM, int SYS>
struct L {
  static void cell(const Grid& g, const double* S, const Work& w, int slot, cudaStream_t st) {
    hw::k_cell<DIM, SYS><<<blocks_for(g.plane), hw::kThreads, 0, st>>>(g, S, w, slot);
  }
  static void face(const Grid& g, const double* S, const Work& w, int slot, cudaStream_t st) {
    const long long nfx = (long long)(g.nx + 1) * g.ny;
    const long long nfy = DIM == 2 ? (long long)(g.ny + 1) * g.nx : 0;
    dim3 grid(blocks_for(nfx > nfy ? nfx : nfy), DIM);
    hw::k_face<DIM, SYS><<<grid, hw::kThreads, 0, st>>>(g, S, w, slot);
  }
  static void update(const Grid& g, double* S, const Work& w, int mode, int stage, double a, double b,
                     double dt, int slot, double* Lo, double* Mo, cudaStream_t st) {
    hw::k_update<DIM, SYS><<<blocks_for(g.plane), hw::kThreads, 0, st>>>(g, S, w, mode, stage, a, b, dt, slot, Lo, Mo);
  }
  static void wavespeed(const Grid& g, const double* S, const Work& w, int slot, cudaStream_t st) {
    hw::k_wavespeed<DIM, SYS><<<blocks_for(g.plane), hw::kThreads, 0, st>>>(g, S, w, slot);
  }
  static constexpr Launchers table() { return Launchers{&cell, &face, &update, &wavespeed}; }
};

const Launchers kTable[2][3] = {
    {L<1, hw::SYS_ADV>::table(), L<1, hw::SYS_BURGERS>::table(), L<1, hw::SYS_EULER>::table()},
    {L<2, hw::SYS_ADV>::table(), L<2, hw::SYS_BURGERS>::table(), L<2, hw::SYS_EULER>::table()}};

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct hweno_ctx {
  int dim, system, bc;
  int64_t nx, ny;
  double dx, dy, gamma;
  double gamma0, d0, eps, cfl, ax, ay;
  cudaStream_t stream;
  double* state;
  unsigned char* ws;
  Work w;
  long long launches;
  // optional per-kernel timing: events recorded around the three launches of every stage
  bool profiling;
  std::vector<cudaEvent_t> events;  // groups of 4: before cell, before face, before update, after
  double kernel_ms[3];
  long long kernel_n[3];
};

namespace {

int nc_of(const hweno_ctx* h) { return h->system == HWENO_EULER ? (h->dim == 1 ? 3 : 4) : 1; }
int nf_of(const hweno_ctx* h) { return h->dim + 1; }
int ng_of(const hweno_ctx* h) { return h->dim == 2 ? 3 : 2; }
int np_of(const hweno_ctx* h) { return h->system == HWENO_EULER ? (h->dim == 2 ? 4 : 3) : 0; }

// workspace sub-buffers in bytes, in layout order
struct Layout {
  size_t B, MD, NOD, PRIM, FX, FY, alpha, scal, status, total;
};

Layout layout_of(const hweno_ctx* h) {
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
  l.total = l.B + l.MD + l.NOD + l.PRIM + l.FX + l.FY + l.alpha + l.scal + l.status;
  return l;
}

Grid grid_of(const hweno_ctx* h) {
  Grid g;
  g.nx = (int)h->nx;
  g.ny = (int)h->ny;
  g.bc = h->bc;
  g.pad_ = 0;
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
  g.G = g.g0 / g1;
  g.cdu = (0.75 - g.d1) / g.d1;
  g.csv = 0.25 / g.d1;
  g.Gd = g.d0 / g.d1;
  const double hs[2] = {h->dx, h->dy};
  for (int d = 0; d < 2; ++d) {
    g.h[d] = hs[d];
    g.ih[d] = 1.0 / hs[d];
    g.chh[d] = hw::DCoef::ch * hs[d];
    g.efih[d] = hw::DCoef::ef / hs[d];
    g.egih[d] = hw::DCoef::eg / hs[d];
    g.hih[d] = 0.5 / hs[d];
  }
  return g;
}

inline int cuda_status() { return cudaGetLastError() == cudaSuccess ? HWENO_OK : HWENO_ECUDA; }

int read_status(hweno_ctx* h) {
  unsigned int st = 0;
  if (cudaMemcpyAsync(&st, h->w.status, sizeof(st), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HWENO_ECUDA;
  return st ? HWENO_ENONPHYS : HWENO_OK;
}

const Launchers& launchers(const hweno_ctx* h) { return kTable[h->dim - 1][h->system]; }

// one spatial-operator evaluation: cell, face; then update in the requested mode
int stage(hweno_ctx* h, const double* S_in, double* S_out, int mode, int st, double dt, int slot, double* Lo,
          double* Mo) {
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
  if (ev[1]) cudaEventRecord(ev[1], h->stream);
  f.face(g, S_in, h->w, slot, h->stream);
  if (ev[2]) cudaEventRecord(ev[2], h->stream);
  f.update(g, S_out, h->w, mode, st, a_k[st], b_k[st], dt, slot, Lo, Mo, h->stream);
  if (ev[3]) cudaEventRecord(ev[3], h->stream);
  h->launches += 3;
  return cuda_status();
}

}  // namespace

extern "C" {

int hweno_create(int dim, int system, int64_t nx, int64_t ny, double dx, double dy, double gamma, int bc,
                 hweno_t** out) {
  if (!out) return HWENO_EINVAL;
  *out = nullptr;
  if (dim != 1 && dim != 2) return HWENO_EINVAL;
  if (system < HWENO_ADVECTION || system > HWENO_EULER) return HWENO_EINVAL;
  if (bc < HWENO_BC_PERIODIC || bc > HWENO_BC_REFLECTIVE) return HWENO_EINVAL;
  if (bc == HWENO_BC_REFLECTIVE) return HWENO_EINVAL;  // reflective walls: not in this build
  if (dim == 1) {
    ny = 1;
    dy = dx;
  }
  if (nx < 5 || ny < 1 || (dim == 2 && ny < 5)) return HWENO_EINVAL;
  if (nx > (1 << 28) || ny > (1 << 28) || nx * ny > ((int64_t)1 << 31)) return HWENO_EINVAL;
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy)) return HWENO_EINVAL;
  if (system == HWENO_EULER && !(gamma > 1.0)) return HWENO_EINVAL;
  hweno_ctx* h = new (std::nothrow) hweno_ctx();
  if (!h) return HWENO_ENOMEM;
  h->dim = dim;
  h->system = system;
  h->bc = bc;
  h->nx = nx;
  h->ny = ny;
  h->dx = dx;
  h->dy = dy;
  h->gamma = system == HWENO_EULER ? gamma : 1.4;
  h->gamma0 = dim == 1 ? 0.95 : 0.99;
  h->d0 = 0.9;
  h->eps = 1e-10;
  h->cfl = 0.6;
  h->ax = 1.0;
  h->ay = 1.0;
  h->stream = nullptr;
  h->state = nullptr;
  h->ws = nullptr;
  h->launches = 0;
  h->profiling = false;
  for (int k = 0; k < 3; ++k) {
    h->kernel_ms[k] = 0.0;
    h->kernel_n[k] = 0;
  }
  *out = h;
  return HWENO_OK;
}

int hweno_set_params(hweno_t* h, double gamma0, double d0, double eps, double cfl, double adv_ax, double adv_ay) {
  if (!h) return HWENO_EINVAL;
  if (!(gamma0 > 0.0 && gamma0 < 1.0) || !(d0 > 0.0 && d0 < 1.0) || !(eps > 0.0) || !(cfl > 0.0))
    return HWENO_EINVAL;
  if (!std::isfinite(adv_ax) || !std::isfinite(adv_ay)) return HWENO_EINVAL;
  h->gamma0 = gamma0;
  h->d0 = d0;
  h->eps = eps;
  h->cfl = cfl;
  h->ax = adv_ax;
  h->ay = adv_ay;
  return HWENO_OK;
}

int hweno_set_stream(hweno_t* h, void* s) {
  if (!h) return HWENO_EINVAL;
  h->stream = static_cast<cudaStream_t>(s);
  return HWENO_OK;
}

size_t hweno_state_doubles(const hweno_t* h) {
  if (!h) return 0;
  return (size_t)nf_of(h) * nc_of(h) * (size_t)h->nx * h->ny;
}

size_t hweno_workspace_bytes(const hweno_t* h) { return h ? layout_of(h).total : 0; }

int hweno_bind(hweno_t* h, double* state_dev, void* ws) {
  if (!h || !state_dev || !ws) return HWENO_EINVAL;
  if (((uintptr_t)state_dev & 15) || ((uintptr_t)ws & 255)) return HWENO_EINVAL;
  const Layout l = layout_of(h);
  unsigned char* p = static_cast<unsigned char*>(ws);
  h->w.B = reinterpret_cast<double*>(p);
  p += l.B;
  h->w.MD = reinterpret_cast<double*>(p);
  p += l.MD;
  h->w.NOD = reinterpret_cast<double*>(p);
  p += l.NOD;
  h->w.PRIM = reinterpret_cast<double*>(p);
  p += l.PRIM;
  h->w.FX = reinterpret_cast<double*>(p);
  p += l.FX;
  h->w.FY = l.FY ? reinterpret_cast<double*>(p) : nullptr;
  p += l.FY;
  h->w.alpha = reinterpret_cast<unsigned long long*>(p);
  unsigned char* scal_begin = p;
  p += l.alpha;
  h->w.scal = reinterpret_cast<double*>(p);
  p += l.scal;
  h->w.status = reinterpret_cast<unsigned int*>(p);
  p += l.status;
  h->state = state_dev;
  h->ws = static_cast<unsigned char*>(ws);
  if (cudaMemsetAsync(scal_begin, 0, l.alpha + l.scal + l.status, h->stream) != cudaSuccess) return HWENO_ECUDA;
  return HWENO_OK;
}

int hweno_rhs(hweno_t* h, const double* S, double* Lo, double* Mo) {
  if (!h || !S || !Lo || !Mo) return HWENO_EINVAL;
  if (!h->ws) return HWENO_ESTATE;
  if (S == Lo || S == Mo || Lo == Mo) return HWENO_EINVAL;
  return stage(h, S, const_cast<double*>(S), 1, 0, 0.0, 3, Lo, Mo);
}

int hweno_step(hweno_t* h, double dt) {
  if (!h) return HWENO_EINVAL;
  if (!h->ws || !h->state) return HWENO_ESTATE;
  if (!std::isfinite(dt)) return HWENO_EINVAL;
  for (int st = 0; st < 3; ++st) {
    int rc = stage(h, h->state, h->state, 0, st, dt, st, nullptr, nullptr);
    if (rc) return rc;
  }
  return HWENO_OK;
}

int hweno_steps(hweno_t* h, double dt, int nsteps) {
  if (!h || nsteps < 0) return HWENO_EINVAL;
  for (int s = 0; s < nsteps; ++s) {
    int rc = hweno_step(h, dt);
    if (rc) return rc;
  }
  return HWENO_OK;
}

int hweno_set_time(hweno_t* h, double t, double t_end) {
  if (!h) return HWENO_EINVAL;
  if (!h->ws) return HWENO_ESTATE;
  if (!std::isfinite(t) || !std::isfinite(t_end)) return HWENO_EINVAL;
  double v[2] = {t, t_end};
  if (cudaMemcpyAsync(h->w.scal + 1, v, sizeof(v), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HWENO_ECUDA;
  return HWENO_OK;
}

int hweno_last_dt(hweno_t* h, double* dt_host, double* t_host) {
  if (!h) return HWENO_EINVAL;
  if (!h->ws) return HWENO_ESTATE;
  double v[2] = {0, 0};
  if (cudaMemcpyAsync(v, h->w.scal, sizeof(v), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  int rc = read_status(h);
  if (dt_host) *dt_host = v[0];
  if (t_host) *t_host = v[1];
  return rc;
}

int hweno_max_wavespeed(hweno_t* h, double* ax, double* ay) {
  if (!h || !ax || !ay) return HWENO_EINVAL;
  if (!h->ws || !h->state) return HWENO_ESTATE;
  if (cudaMemsetAsync(h->w.alpha + 6, 0, 2 * sizeof(unsigned long long), h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  launchers(h).wavespeed(grid_of(h), h->state, h->w, 3, h->stream);
  h->launches += 1;
  if (cuda_status()) return HWENO_ECUDA;
  unsigned long long bits[2] = {0, 0};
  if (cudaMemcpyAsync(bits, h->w.alpha + 6, sizeof(bits), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  int rc = read_status(h);
  double a, b;
  std::memcpy(&a, &bits[0], 8);
  std::memcpy(&b, &bits[1], 8);
  *ax = a;
  *ay = h->dim == 2 ? b : 0.0;
  return rc;
}

int hweno_sync(hweno_t* h) {
  if (!h) return HWENO_EINVAL;
  if (!h->ws) {
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? HWENO_OK : HWENO_ECUDA;
  }
  return read_status(h);
}

int hweno_upload(hweno_t* h, const double* host) {
  if (!h || !host) return HWENO_EINVAL;
  if (!h->state) return HWENO_ESTATE;
  if (cudaMemcpyAsync(h->state, host, hweno_state_doubles(h) * 8, cudaMemcpyHostToDevice, h->stream) !=
      cudaSuccess)
    return HWENO_ECUDA;
  return HWENO_OK;
}

int hweno_download(hweno_t* h, double* host) {
  if (!h || !host) return HWENO_EINVAL;
  if (!h->state) return HWENO_ESTATE;
  if (cudaMemcpyAsync(host, h->state, hweno_state_doubles(h) * 8, cudaMemcpyDeviceToHost, h->stream) !=
      cudaSuccess)
    return HWENO_ECUDA;
  return HWENO_OK;
}

int hweno_set_profiling(hweno_t* h, int on) {
  if (!h) return HWENO_EINVAL;
  h->profiling = on != 0;
  return HWENO_OK;
}

int hweno_kernel_times(hweno_t* h, double* ms3, long long* n3) {
  if (!h || !ms3 || !n3) return HWENO_EINVAL;
  if (!h->events.empty()) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HWENO_ECUDA;
    for (size_t b = 0; b + 3 < h->events.size(); b += 4) {
      for (int k = 0; k < 3; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->events[b + k], h->events[b + k + 1]) != cudaSuccess) return HWENO_ECUDA;
        h->kernel_ms[k] += ms;
        h->kernel_n[k] += 1;
      }
    }
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    h->events.clear();
  }
  for (int k = 0; k < 3; ++k) {
    ms3[k] = h->kernel_ms[k];
    n3[k] = h->kernel_n[k];
    h->kernel_ms[k] = 0.0;
    h->kernel_n[k] = 0;
  }
  return HWENO_OK;
}

void hweno_destroy(hweno_t* h) {
  if (!h) return;
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  delete h;
}

const char* hweno_strerror(int s) {
  switch (s) {
    case HWENO_OK: return "ok";
    case HWENO_EINVAL: return "invalid argument";
    case HWENO_ECUDA: return "CUDA error";
    case HWENO_ENOMEM: return "out of memory or workspace too small";
    case HWENO_ENONPHYS: return "non-physical state (rho <= 0, P <= 0 or non-finite wavespeed)";
    case HWENO_ESTATE: return "call out of order (no state or workspace bound)";
    case HWENO_ETOOBIG: return "grid too large for the fixed device scratch of hweno_rhs_static (16 MiB)";
    default: return "unknown status";
  }
}

long long hweno_launch_count(const hweno_t* h) { return h ? h->launches : -1; }

int hweno_selftest_rcp(const double* x_dev, double* r_dev, int64_t n, void* stream) {
  if (!x_dev || !r_dev || n < 0) return HWENO_EINVAL;
  if (n == 0) return HWENO_OK;
  hw::k_rcp_check<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x_dev, r_dev, n);
  return cuda_status();
}

}  // extern "C"

// =============================================================================================
// hweno_rhs_static: the spatial operator without any allocation.
//
// Some callers cannot allocate device memory for a workspace: host programs that hand a library
// only the input and output buffers because a framework or memory pool of their own owns every
// device allocation, and latency-sensitive loops in which a cudaMalloc (which can synchronise the
// whole device) is not acceptable.  For them this entry point runs the same three kernels as
// hweno_rhs but takes its scratch (modified derivatives, nodal values, primitives, face fluxes,
// wavespeed slot and status word) from the fixed array below, which every GPU that loads this
// library holds until the process exits.
namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// device address of g_static_scratch, looked up once per device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory)
std::atomic<void*> g_static_scratch_dev[kMaxDevices];

int static_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HWENO_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return HWENO_ECUDA;
  void* p = g_static_scratch_dev[dev].load(std::memory_order_acquire);
  if (!p) {
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HWENO_ECUDA;
    g_static_scratch_dev[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return HWENO_OK;
}

}  // namespace

extern "C" int hweno_rhs_static(int dim, int system, int64_t nx, int64_t ny, double dx, double dy, double gamma,
                                int bc, const double* params5, const double* S, double* Lo, double* Mo,
                                void* stream) {
  if (!S || !Lo || !Mo || S == Lo || S == Mo || Lo == Mo) return HWENO_EINVAL;
  // the same validation as hweno_create, on a handle that lives on this stack frame
  hweno_ctx h;
  if (dim != 1 && dim != 2) return HWENO_EINVAL;
  if (system < HWENO_ADVECTION || system > HWENO_EULER) return HWENO_EINVAL;
  if (bc < HWENO_BC_PERIODIC || bc > HWENO_BC_REFLECTIVE || bc == HWENO_BC_REFLECTIVE) return HWENO_EINVAL;
  if (dim == 1) {
    ny = 1;
    dy = dx;
  }
  if (nx < 5 || ny < 1 || (dim == 2 && ny < 5)) return HWENO_EINVAL;
  if (nx > (1 << 28) || ny > (1 << 28)) return HWENO_ETOOBIG;
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy)) return HWENO_EINVAL;
  if (system == HWENO_EULER && !(gamma > 1.0)) return HWENO_EINVAL;
  h.dim = dim;
  h.system = system;
  h.bc = bc;
  h.nx = nx;
  h.ny = ny;
  h.dx = dx;
  h.dy = dy;
  h.gamma = system == HWENO_EULER ? gamma : 1.4;
  h.gamma0 = dim == 1 ? 0.95 : 0.99;
  h.d0 = 0.9;
  h.eps = 1e-10;
  h.cfl = 0.6;
  h.ax = 1.0;
  h.ay = 1.0;
  if (params5) {
    if (!(params5[0] > 0.0 && params5[0] < 1.0) || !(params5[1] > 0.0 && params5[1] < 1.0) || !(params5[2] > 0.0) ||
        !std::isfinite(params5[3]) || !std::isfinite(params5[4]))
      return HWENO_EINVAL;
    h.gamma0 = params5[0];
    h.d0 = params5[1];
    h.eps = params5[2];
    h.ax = params5[3];
    h.ay = params5[4];
  }
  h.stream = static_cast<cudaStream_t>(stream);
  h.state = nullptr;
  h.ws = nullptr;
  h.launches = 0;
  h.profiling = false;
  // scratch layout: the workspace layout of hweno_bind without the stage base B
  const Layout l = layout_of(&h);
  const size_t need = l.total - l.B;
  if (need > kStaticScratchBytes) return HWENO_ETOOBIG;
  void* base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);
  h.w.B = nullptr;  // not used by the rhs mode
  h.w.MD = reinterpret_cast<double*>(p);
  p += l.MD;
  h.w.NOD = reinterpret_cast<double*>(p);
  p += l.NOD;
  h.w.PRIM = reinterpret_cast<double*>(p);
  p += l.PRIM;
  h.w.FX = reinterpret_cast<double*>(p);
  p += l.FX;
  h.w.FY = l.FY ? reinterpret_cast<double*>(p) : nullptr;
  p += l.FY;
  h.w.alpha = reinterpret_cast<unsigned long long*>(p);
  unsigned char* scal_begin = p;
  p += l.alpha;
  h.w.scal = reinterpret_cast<double*>(p);
  p += l.scal;
  h.w.status = reinterpret_cast<unsigned int*>(p);
  // the array keeps the previous call's contents: clear the wavespeed slots and the status word
  if (cudaMemsetAsync(scal_begin, 0, l.alpha + l.scal + l.status, h.stream) != cudaSuccess) return HWENO_ECUDA;
  return stage(&h, S, const_cast<double*>(S), 1, 0, 0.0, 3, Lo, Mo);
}
