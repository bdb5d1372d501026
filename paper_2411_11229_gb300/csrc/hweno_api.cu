// C ABI of libhweno.so: see include/hweno.h for the contract of every entry point.
#include "hweno_host.cuh"

using namespace hwh;

namespace hw {
// applies the library's FP64 reciprocal to n values (accuracy self-test)
__global__ void k_rcp_check(const double* __restrict__ x, double* __restrict__ r, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = rcp(x[i]);
}

// FP64 issue probe: kDfmaChains independent chains a <- a b + c per thread, kDfmaIters times.  b
// and c are read from a per-thread address (p[0] = p[1] = b, p[2] = p[3] = c), so they live in
// thread registers, the operand form of the stage kernels' DFMAs.  The chains' sum is stored only
// if it equals p[0] exactly, which the data (b just below 1, c small and positive) never give; the
// store keeps the chains live.
constexpr int kDfmaChains = 8, kDfmaIters = 2048, kDfmaThreads = 256, kDfmaBlocksPerSM = 8;
__global__ void __launch_bounds__(kDfmaThreads) k_dfma_probe(double* __restrict__ p) {
  const double b = p[threadIdx.x & 1], c = p[2 + (threadIdx.x & 1)];
  double a[kDfmaChains];
#pragma unroll
  for (int k = 0; k < kDfmaChains; ++k) a[k] = 0.5 + 0.01 * k + 1e-6 * threadIdx.x;
#pragma unroll 4
  for (int it = 0; it < kDfmaIters; ++it)
#pragma unroll
    for (int k = 0; k < kDfmaChains; ++k) a[k] = fma(a[k], b, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kDfmaChains; ++k) s += a[k];
  if (s == p[0]) p[3] = s;
}

#ifdef HWENO_BOUNDS_CHECK
// self-test of the bounds check: the check applied to an index one past the end of a two-element
// array; the kernel then writes element 0 (a constant index), whatever the check returned
__device__ double g_bounds_probe[2];
__global__ void k_bounds_probe(long long n) {
  const long long i = HW_IDX(n, n);
  g_bounds_probe[0] = (double)i;
}
#endif
}  // namespace hw

namespace {
// the scheme of the paper with one boundary type on every side
void set_plain_scheme(hweno_ctx* h, int bc) {
  h->var = 0;
  h->flags = 0;
  h->grav = 0.0;
  for (int sd = 0; sd < 4; ++sd) {
    h->side[sd] = bc;
    for (int k = 0; k < 4; ++k) h->fixed[sd][k] = 0.0;
  }
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
  if (bc == HWENO_BC_REFLECTIVE && system != HWENO_EULER) return HWENO_EINVAL;  // sign tables: Euler only
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
  set_plain_scheme(h, bc);
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

int hweno_create_ex(int dim, int system, int64_t nx, int64_t ny, double dx, double dy, double gamma,
                    const hweno_ext* ext, hweno_t** out) {
  if (!out) return HWENO_EINVAL;
  *out = nullptr;
  if (!ext) return HWENO_EINVAL;
  const int nsides = dim == 2 ? 4 : 2;
  for (int sd = 0; sd < nsides; ++sd) {
    const int t = ext->side[sd];
    if (t < HWENO_BC_PERIODIC || t > HWENO_BC_FIXED) return HWENO_EINVAL;
    if (t == HWENO_BC_REFLECTIVE && system != HWENO_EULER) return HWENO_EINVAL;
  }
  // periodic pairs the two ends of an axis
  if ((ext->side[0] == HWENO_BC_PERIODIC) != (ext->side[1] == HWENO_BC_PERIODIC)) return HWENO_EINVAL;
  if (dim == 2 && (ext->side[2] == HWENO_BC_PERIODIC) != (ext->side[3] == HWENO_BC_PERIODIC)) return HWENO_EINVAL;
  const int all_flags = HWENO_FLAG_V_WEIGHTED | HWENO_FLAG_CD2 | HWENO_FLAG_R2 | HWENO_FLAG_ALPHA_STEP |
                        HWENO_FLAG_ALPHA_LOCAL;
  if (ext->flags < 0 || (ext->flags & ~all_flags)) return HWENO_EINVAL;
  if (!std::isfinite(ext->grav)) return HWENO_EINVAL;
  if (ext->grav != 0.0 && !(dim == 2 && system == HWENO_EULER)) return HWENO_EINVAL;
  const int nc = system == HWENO_EULER ? (dim == 1 ? 3 : 4) : 1;
  bool uniform = true, any_fixed = false;
  for (int sd = 0; sd < nsides; ++sd) {
    uniform = uniform && ext->side[sd] == ext->side[0];
    if (ext->side[sd] != HWENO_BC_FIXED) continue;
    any_fixed = true;
    const double* U = ext->fixed[sd];
    for (int k = 0; k < nc; ++k)
      if (!std::isfinite(U[k])) return HWENO_EINVAL;
    if (system == HWENO_EULER) {
      const double vv = dim == 2 ? U[1] * U[1] + U[2] * U[2] : U[1] * U[1];
      if (!(U[0] > 0.0) || !((gamma - 1.0) * (U[nc - 1] - 0.5 * vv / U[0]) > 0.0)) return HWENO_EINVAL;
    }
  }
  const int bc0 = any_fixed ? HWENO_BC_TRANSMISSIVE : ext->side[0];
  int rc = hweno_create(dim, system, nx, ny, dx, dy, gamma, bc0, out);
  if (rc) return rc;
  hweno_ctx* h = *out;
  h->flags = ext->flags;
  h->grav = ext->grav;
  for (int sd = 0; sd < 4; ++sd) {
    h->side[sd] = sd < nsides ? ext->side[sd] : HWENO_BC_PERIODIC;
    for (int k = 0; k < 4; ++k) h->fixed[sd][k] = k < nc ? ext->fixed[sd][k] : 0.0;
  }
  // the scheme of the paper with one boundary type runs the plain kernels
  const bool plain = ext->flags == 0 && ext->grav == 0.0 && uniform && !any_fixed;
  h->var = plain ? 0 : ((ext->flags & HWENO_FLAG_R2) && system == HWENO_EULER ? 2 : 1);
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
  h->w.astride = 2;
  p += l.status;
  h->w.FS = l.FS ? reinterpret_cast<double*>(p) : nullptr;
  p += l.FS;
  h->w.GFS = l.GFS ? reinterpret_cast<double*>(p) : nullptr;
  p += l.GFS;
  h->w.gstride = gstride_of(h);
  h->w.WS = l.WS ? reinterpret_cast<double*>(p) : nullptr;
  p += l.WS;
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
  double v[3] = {t, t_end, 0.0};  // time, end time, steps taken
  if (cudaMemcpyAsync(h->w.scal + 1, v, sizeof(v), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return HWENO_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return HWENO_ECUDA;
  return HWENO_OK;
}

int hweno_run(hweno_t* h, double t_end, int64_t max_steps, int64_t* steps_done) {
  if (!h || !(t_end > 0.0) || !std::isfinite(t_end) || max_steps < 0) return HWENO_EINVAL;
  if (!h->ws || !h->state) return HWENO_ESTATE;
  if (steps_done) *steps_done = 0;
  int rc = hweno_set_time(h, 0.0, t_end);
  if (rc) return rc;
  constexpr int kChunk = 16;  // CFL steps issued between two looks at the device clock
  // Record one chunk as a CUDA graph on a private stream (the handle's stream may be the legacy
  // default stream, which cannot be captured); steps past the end time leave the state unchanged,
  // so a whole chunk can be issued without knowing where in it the end time falls.
  cudaStream_t user = h->stream, priv = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  long long chunk_launches = 0;
  if (!h->profiling && max_steps >= kChunk &&
      cudaStreamCreateWithFlags(&priv, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess) {
    h->stream = priv;
    const long long l0 = h->launches;
    cudaGraph_t gr = nullptr;
    bool ok = cudaStreamBeginCapture(priv, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      for (int k = 0; k < kChunk && ok; ++k)
        for (int st = 0; st < 3 && ok; ++st) ok = stage(h, h->state, h->state, 0, st, 0.0, st, nullptr, nullptr) == HWENO_OK;
      const bool ended = cudaStreamEndCapture(priv, &gr) == cudaSuccess;
      ok = ok && ended && gr;
    }
    chunk_launches = h->launches - l0;
    h->launches = l0;
    if (!ok || cudaGraphInstantiate(&exec, gr, 0) != cudaSuccess) exec = nullptr;
    if (gr) cudaGraphDestroy(gr);
    h->stream = user;
    cudaGetLastError();  // a failed capture leaves the plain path
  }
  rc = HWENO_OK;
  for (;;) {
    double v[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(v, h->w.scal, sizeof(v), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) {
      rc = HWENO_ECUDA;
      break;
    }
    rc = read_status(h);  // synchronises
    if (rc) break;
    const int64_t done = (int64_t)v[3];
    if (steps_done) *steps_done = done;
    if (!std::isfinite(v[1])) {
      rc = HWENO_ENONPHYS;
      break;
    }
    if (v[1] >= t_end || done >= max_steps) break;
    const int64_t left = max_steps - done;
    if (exec && left >= kChunk) {
      if (cudaEventRecord(fork, user) != cudaSuccess || cudaStreamWaitEvent(priv, fork, 0) != cudaSuccess ||
          cudaGraphLaunch(exec, priv) != cudaSuccess || cudaEventRecord(join, priv) != cudaSuccess ||
          cudaStreamWaitEvent(user, join, 0) != cudaSuccess) {
        rc = HWENO_ECUDA;
        break;
      }
      h->launches += chunk_launches;
    } else {
      for (int64_t k = 0; k < (left < kChunk ? left : kChunk) && !rc; ++k) rc = hweno_step(h, 0.0);
      if (rc) break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (priv) {
    cudaStreamSynchronize(priv);
    cudaStreamDestroy(priv);
  }
  return rc;
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

size_t hweno_pipeline_slot_bytes(const hweno_t* h) {
  if (!h) return 0;
  return align_up(hweno_state_doubles(h) * 8) + hweno_workspace_bytes(h);
}

int hweno_pipeline(hweno_t* h, int count, const double* const* host_in, double* const* host_out, int nsteps,
                   int depth, void* slot_mem) {
  if (!h || count < 0 || nsteps < 0 || depth < 1 || depth > 8 || !slot_mem) return HWENO_EINVAL;
  if ((uintptr_t)slot_mem & 255) return HWENO_EINVAL;
  if (count > 0 && (!host_in || !host_out)) return HWENO_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!host_in[i] || !host_out[i]) return HWENO_EINVAL;
  const size_t bytes = hweno_state_doubles(h) * 8, sb = align_up(bytes), per = hweno_pipeline_slot_bytes(h);
  unsigned char* base = static_cast<unsigned char*>(slot_mem);
  // the slots: copies of the handle's scheme, each bound to its own state and workspace and
  // launching on its own stream, ordered after the work already queued on the handle's stream
  std::vector<hweno_ctx> slot(depth, *h);
  std::vector<cudaStream_t> st(depth, nullptr);
  cudaEvent_t start = nullptr;
  int rc = cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess &&
                   cudaEventRecord(start, h->stream) == cudaSuccess
               ? HWENO_OK
               : HWENO_ECUDA;
  for (int d = 0; d < depth && !rc; ++d) {
    hweno_ctx& s = slot[d];
    s.events.clear();
    s.profiling = false;
    s.launches = 0;
    if (cudaStreamCreateWithFlags(&st[d], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(st[d], start, 0) != cudaSuccess) {
      rc = HWENO_ECUDA;
      break;
    }
    s.stream = st[d];
    rc = hweno_bind(&s, reinterpret_cast<double*>(base + d * per), base + d * per + sb);
  }
  // problem i on slot i mod depth: upload, nsteps CFL steps, download, in that slot's stream order
  for (int i = 0; i < count && !rc; ++i) {
    hweno_ctx& s = slot[i % depth];
    if (cudaMemcpyAsync(s.state, host_in[i], bytes, cudaMemcpyHostToDevice, s.stream) != cudaSuccess) {
      rc = HWENO_ECUDA;
      break;
    }
    for (int k = 0; k < nsteps && !rc; ++k) rc = hweno_step(&s, 0.0);
    if (!rc && cudaMemcpyAsync(host_out[i], s.state, bytes, cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
      rc = HWENO_ECUDA;
  }
  // wait for every slot; the handle's stream is ordered after them
  for (int d = 0; d < depth; ++d) {
    if (!st[d]) continue;
    const int sr = read_status(&slot[d]);  // synchronises the slot's stream
    if (!rc) rc = sr;
    h->launches += slot[d].launches;
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done, st[d]);
      cudaStreamWaitEvent(h->stream, done, 0);
      cudaEventDestroy(done);
    }
    cudaStreamDestroy(st[d]);
  }
  if (start) cudaEventDestroy(start);
  return rc;
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

int hweno_selftest_fp64_peak(double* scratch_dev, int reps, void* stream, double* dfma_per_s,
                             double* dfma_per_launch) {
  if (!scratch_dev || !dfma_per_s || reps < 1 || reps > 100) return HWENO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return HWENO_ECUDA;
  // b just below 1 and c small: the chains converge to c / (1 - b) = 1e3 and stay finite
  const double ops[4] = {0.999999, 0.999999, 1e-3, 1e-3};
  if (cudaMemcpyAsync(scratch_dev, ops, sizeof(ops), cudaMemcpyHostToDevice, st) != cudaSuccess) return HWENO_ECUDA;
  const unsigned blocks = (unsigned)sms * hw::kDfmaBlocksPerSM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return HWENO_ECUDA;
  }
  int rc = HWENO_OK;
  float best = 0.0f;
  hw::k_dfma_probe<<<blocks, hw::kDfmaThreads, 0, st>>>(scratch_dev);  // untimed
  for (int r = 0; r < reps && rc == HWENO_OK; ++r) {
    float ms = 0.0f;
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = HWENO_ECUDA;
    hw::k_dfma_probe<<<blocks, hw::kDfmaThreads, 0, st>>>(scratch_dev);
    if (rc == HWENO_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                           cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = HWENO_ECUDA;
    if (rc == HWENO_OK && (best == 0.0f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  const double per_launch = (double)blocks * hw::kDfmaThreads * hw::kDfmaIters * hw::kDfmaChains;
  *dfma_per_s = best > 0.0f ? per_launch / (best * 1e-3) : 0.0;
  if (dfma_per_launch) *dfma_per_launch = per_launch;
  return HWENO_OK;
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
  set_plain_scheme(&h, bc);
  if (dim != 1 && dim != 2) return HWENO_EINVAL;
  if (system < HWENO_ADVECTION || system > HWENO_EULER) return HWENO_EINVAL;
  if (bc < HWENO_BC_PERIODIC || bc > HWENO_BC_REFLECTIVE) return HWENO_EINVAL;
  if (bc == HWENO_BC_REFLECTIVE && system != HWENO_EULER) return HWENO_EINVAL;
  if (dim == 1) {
    ny = 1;
    dy = dx;
  }
  if (nx < 5 || ny < 1 || (dim == 2 && ny < 5)) return HWENO_EINVAL;
  // every cell needs more than 8 bytes of scratch: a grid with more cells than the array holds
  // doubles is refused here, before the layout's byte counts are formed (they cannot overflow)
  if (nx > (1 << 28) || ny > (1 << 28) || nx * ny > (int64_t)(kStaticScratchBytes / 8)) return HWENO_ETOOBIG;
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
  h.w.astride = 2;
  h.w.FS = h.w.GFS = h.w.WS = nullptr;
  h.w.gstride = 0;
  // the array keeps the previous call's contents: clear the wavespeed slots and the status word
  if (cudaMemsetAsync(scal_begin, 0, l.alpha + l.scal + l.status, h.stream) != cudaSuccess) return HWENO_ECUDA;
  return stage(&h, S, const_cast<double*>(S), 1, 0, 0.0, 3, Lo, Mo);
}

extern "C" long long hweno_bounds_status(int* where) {
#ifdef HWENO_BOUNDS_CHECK
  if (cudaDeviceSynchronize() != cudaSuccess) return HWENO_ECUDA;
  int l0 = 0, l1 = 0, l2 = 0;
  const unsigned int c0 = hw::bounds_take(&l0), c1 = hwh::bounds_take_batch(&l1), c2 = hwh::bounds_take_adjoint(&l2);
  if (where) *where = c0 ? l0 : (c1 ? 100000 + l1 : (c2 ? 200000 + l2 : 0));
  return (long long)c0 + c1 + c2;
#else
  if (where) *where = 0;
  return -1;
#endif
}

extern "C" long long hweno_bounds_selftest(void) {
#ifdef HWENO_BOUNDS_CHECK
  const long long before = hweno_bounds_status(nullptr);
  if (before < 0) return before;
  hw::k_bounds_probe<<<1, 1>>>(2);
  if (cudaGetLastError() != cudaSuccess) return HWENO_ECUDA;
  return hweno_bounds_status(nullptr);
#else
  return -1;
#endif
}
