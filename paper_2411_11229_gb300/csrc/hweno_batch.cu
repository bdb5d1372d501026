// Batched HWENO-I: many independent Euler problems of uneven sizes (1D lines and 2D grids)
// advanced together.  See include/hweno.h (hweno_batch_*) for the contract.
//
// A batched stage runs over a work-list of tiles of all instances, in one of two launch shapes
// chosen by the autotuner: ONE persistent cooperative launch (phase 1 the cell work of every
// tile: wavespeeds into per-instance slots, nodal values, modified derivatives; a grid barrier;
// phase 2 the face work; a grid barrier; phase 3 the conservative update with a per-instance CFL
// step), or the same three phases as three persistent launches, each at its own register budget.
// The stages of a step are recorded once in a CUDA graph and replayed.  The comparison path
// launches the three single-grid kernels per instance and stage.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>

#include "hweno_host.cuh"

namespace cg = cooperative_groups;
using namespace hwh;

namespace hw {

struct BatchInst {
  Grid g;
  Work w;
  double* S;
  int dim;
  int pad_;
};

// work items: (instance, first tile) for cells; (instance, direction, first tile) for faces
struct BatchArgs {
  const BatchInst* inst;
  const int2* cells;
  const int4* faces;
  int ncells, nfaces, tiles_per_item, ninst;
  int ncells2, nfaces2;  // the work-list holds the 2D items first: [0, n*2) 2D, [n*2, n) 1D
  int stage;
  double a_k, b_k;
  int slot;
};

template <int DIM>
__device__ __forceinline__ void batch_cells(const BatchInst& I, long long p0, int tpi, int slot) {
  double wsx = 0.0, wsy = 0.0;
  for (int t = 0; t < tpi; ++t) {
    const long long p = p0 + (long long)t * kThreads + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (p < I.g.plane) cell_body<DIM, SYS_EULER>(I.g, I.S, I.w, p, a, b);
    wsx = fmax(wsx, a);
    wsy = fmax(wsy, b);
  }
  block_max2(wsx, wsy, I.w.alpha + slot * I.w.astride);
  __syncthreads();  // the reduction's shared arrays are reused by the next item
}

template <int DIM>
__device__ __forceinline__ void batch_faces(const BatchInst& I, int dir, long long f0, int tpi, int slot) {
  const long long nf = dir == 0 ? (long long)(I.g.nx + 1) * I.g.ny : (long long)(I.g.ny + 1) * I.g.nx;
  const double alpha = __longlong_as_double((long long)I.w.alpha[slot * I.w.astride + dir]);
  for (int t = 0; t < tpi; ++t) {
    const long long f = f0 + (long long)t * kThreads + threadIdx.x;
    if (f < nf) face_body<DIM, SYS_EULER>(I.g, I.S, I.w, dir, f, alpha);
  }
}

template <int DIM>
__device__ __forceinline__ void batch_update(const BatchInst& I, long long p0, int tpi, const BatchArgs& a) {
  const double dt = stage_dt<DIM>(I.g, I.w, a.stage, 0.0, a.slot);
  if (a.stage == 0 && p0 == 0 && threadIdx.x == 0) I.w.scal[0] = dt;
  if (dt == 0.0) return;  // the instance has reached its end time
  for (int t = 0; t < tpi; ++t) {
    const long long p = p0 + (long long)t * kThreads + threadIdx.x;
    if (p < I.g.plane) update_body<DIM, SYS_EULER>(I.g, I.S, I.w, 0, a.stage, a.a_k, a.b_k, dt, p, nullptr, nullptr);
  }
  if (a.stage == 2 && p0 == 0 && threadIdx.x == 0) {
    I.w.scal[1] += dt;
    I.w.scal[3] += 1.0;
  }
}

// One Runge-Kutta stage of every instance.  Launched cooperatively with every block resident.
__global__ void __launch_bounds__(kThreads) k_batch_stage(BatchArgs a) {
  cg::grid_group grid = cg::this_grid();
  const long long span = (long long)kThreads * a.tiles_per_item;
  for (int it = blockIdx.x; it < a.ncells; it += gridDim.x) {
    const int2 c = a.cells[it];
    const BatchInst& I = a.inst[HW_IDX(c.x, a.ninst)];
    if (I.dim == 1)
      batch_cells<1>(I, c.y * span, a.tiles_per_item, a.slot);
    else
      batch_cells<2>(I, c.y * span, a.tiles_per_item, a.slot);
  }
  grid.sync();
  for (int it = blockIdx.x; it < a.nfaces; it += gridDim.x) {
    const int4 f = a.faces[it];
    const BatchInst& I = a.inst[HW_IDX(f.x, a.ninst)];
    if (I.dim == 1)
      batch_faces<1>(I, 0, f.z * span, a.tiles_per_item, a.slot);
    else
      batch_faces<2>(I, f.y, f.z * span, a.tiles_per_item, a.slot);
  }
  grid.sync();
  for (int it = blockIdx.x; it < a.ncells; it += gridDim.x) {
    const int2 c = a.cells[it];
    const BatchInst& I = a.inst[HW_IDX(c.x, a.ninst)];
    if (I.dim == 1)
      batch_update<1>(I, c.y * span, a.tiles_per_item, a);
    else
      batch_update<2>(I, c.y * span, a.tiles_per_item, a);
  }
}

// The same stage as persistent launches per phase and dimension (cell, face and update work of
// the 2D items, then of the 1D items), each kernel at the register budget of its own code path;
// stream order replaces the grid barriers.
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_batch_cells(BatchArgs a) {
  const long long span = (long long)kThreads * a.tiles_per_item;
  const int lo = DIM == 2 ? 0 : a.ncells2, hi = DIM == 2 ? a.ncells2 : a.ncells;
  for (int it = lo + blockIdx.x; it < hi; it += gridDim.x) {
    const int2 c = a.cells[it];
    batch_cells<DIM>(a.inst[HW_IDX(c.x, a.ninst)], c.y * span, a.tiles_per_item, a.slot);
  }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads, 3) k_batch_faces(BatchArgs a) {
  const long long span = (long long)kThreads * a.tiles_per_item;
  const int lo = DIM == 2 ? 0 : a.nfaces2, hi = DIM == 2 ? a.nfaces2 : a.nfaces;
  for (int it = lo + blockIdx.x; it < hi; it += gridDim.x) {
    const int4 f = a.faces[it];
    batch_faces<DIM>(a.inst[HW_IDX(f.x, a.ninst)], DIM == 2 ? f.y : 0, f.z * span, a.tiles_per_item, a.slot);
  }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_batch_update(BatchArgs a) {
  const long long span = (long long)kThreads * a.tiles_per_item;
  const int lo = DIM == 2 ? 0 : a.ncells2, hi = DIM == 2 ? a.ncells2 : a.ncells;
  for (int it = lo + blockIdx.x; it < hi; it += gridDim.x) {
    const int2 c = a.cells[it];
    batch_update<DIM>(a.inst[HW_IDX(c.x, a.ninst)], c.y * span, a.tiles_per_item, a);
  }
}

}  // namespace hw

namespace hwh {
unsigned int bounds_take_batch(int* line) {
#ifdef HWENO_BOUNDS_CHECK
  return hw::bounds_take(line);
#else
  if (line) *line = 0;
  return 0;
#endif
}
}  // namespace hwh

struct hweno_batch {
  int n;
  std::vector<hweno_ctx> inst;        // per-instance parameters and device views
  std::vector<size_t> state_off;      // offset of instance i in the packed state (doubles)
  size_t state_total;
  std::vector<size_t> ws_off;         // offset of instance i's workspace (bytes)
  size_t ws_inst_total, ws_tables, ws_total;
  cudaStream_t stream;
  double* state;
  unsigned char* ws;
  unsigned long long* alpha;          // [4 slots][n][2]
  hw::BatchInst* d_inst;
  int2* d_cells;
  int4* d_faces;
  int ncells, nfaces;
  int tiles_per_item, blocks_per_sm, max_blocks_per_sm, num_sms;
  int mode;                           // 0: one cooperative launch per stage; 1: three phase launches
  int occ_phase[2][3];                // resident blocks per SM of the phase kernels [1D, 2D][phase]
  int ncells2, nfaces2;               // 2D items come first in the work-lists
  cudaGraphExec_t graph;
  bool graph_ok;
  long long graph_launches;  // kernel launches recorded in the graph of one step
  long long launches;
};

namespace {

constexpr int kMaxTilesPerItem = 4;

int build_items(hweno_batch* b, std::vector<int2>& cells, std::vector<int4>& faces) {
  const long long span = (long long)hw::kThreads * b->tiles_per_item;
  // larger instances first: the grid-stride loop then ends each phase on small items
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (b->inst[x].dim != b->inst[y].dim) return b->inst[x].dim > b->inst[y].dim;  // 2D first
    return b->inst[x].nx * b->inst[x].ny > b->inst[y].nx * b->inst[y].ny;
  });
  cells.clear();
  faces.clear();
  b->ncells2 = b->nfaces2 = 0;
  for (int i : order) {
    const hweno_ctx& h = b->inst[i];
    const long long plane = h.nx * h.ny;
    for (long long t = 0; t * span < plane; ++t) cells.push_back(make_int2(i, (int)t));
    const long long nfx = (h.nx + 1) * h.ny;
    for (long long t = 0; t * span < nfx; ++t) faces.push_back(make_int4(i, 0, (int)t, 0));
    if (h.dim == 2) {
      const long long nfy = (h.ny + 1) * h.nx;
      for (long long t = 0; t * span < nfy; ++t) faces.push_back(make_int4(i, 1, (int)t, 0));
      b->ncells2 = (int)cells.size();
      b->nfaces2 = (int)faces.size();
    }
  }
  return HWENO_OK;
}

int upload_items(hweno_batch* b) {
  std::vector<int2> cells;
  std::vector<int4> faces;
  build_items(b, cells, faces);
  b->ncells = (int)cells.size();
  b->nfaces = (int)faces.size();
  if (cudaMemcpyAsync(b->d_cells, cells.data(), cells.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_faces, faces.data(), faces.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess)
    return HWENO_ECUDA;
  // the host vectors must outlive the asynchronous copies
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return HWENO_ECUDA;
  return HWENO_OK;
}

void drop_graph(hweno_batch* b) {
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  b->graph_ok = false;
}

int launch_stage(hweno_batch* b, int st) {
  static const double a_k[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double b_k[3] = {1.0, 0.25, 2.0 / 3.0};
  if (cudaMemsetAsync(b->alpha + (size_t)st * 2 * b->n, 0, 2 * b->n * sizeof(unsigned long long), b->stream) !=
      cudaSuccess)
    return HWENO_ECUDA;
  hw::BatchArgs a;
  a.inst = b->d_inst;
  a.cells = b->d_cells;
  a.faces = b->d_faces;
  a.ncells = b->ncells;
  a.nfaces = b->nfaces;
  a.tiles_per_item = b->tiles_per_item;
  a.ninst = b->n;
  a.ncells2 = b->ncells2;
  a.nfaces2 = b->nfaces2;
  a.stage = st;
  a.a_k = a_k[st];
  a.b_k = b_k[st];
  a.slot = st;
  if (b->mode == 1) {
    const int items[2][3] = {{b->ncells - b->ncells2, b->nfaces - b->nfaces2, b->ncells - b->ncells2},
                             {b->ncells2, b->nfaces2, b->ncells2}};
    void (*kern[2][3])(hw::BatchArgs) = {
        {hw::k_batch_cells<1>, hw::k_batch_faces<1>, hw::k_batch_update<1>},
        {hw::k_batch_cells<2>, hw::k_batch_faces<2>, hw::k_batch_update<2>}};
    for (int ph = 0; ph < 3; ++ph)
      for (int d = 1; d >= 0; --d) {
        if (items[d][ph] == 0) continue;
        const int grid = std::max(1, std::min(items[d][ph], b->num_sms * b->occ_phase[d][ph]));
        kern[d][ph]<<<grid, hw::kThreads, 0, b->stream>>>(a);
        b->launches += 1;
      }
    if (cudaGetLastError() != cudaSuccess) return HWENO_ECUDA;
    return HWENO_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(b->num_sms * b->blocks_per_sm));
  cfg.blockDim = dim3(hw::kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, hw::k_batch_stage, a) != cudaSuccess) return HWENO_ECUDA;
  b->launches += 1;
  return HWENO_OK;
}

int step_direct(hweno_batch* b) {
  for (int st = 0; st < 3; ++st) {
    int rc = launch_stage(b, st);
    if (rc) return rc;
  }
  return HWENO_OK;
}

// record the three stages of a step once; replay later
int build_graph(hweno_batch* b) {
  drop_graph(b);
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HWENO_ECUDA;
  const long long launches = b->launches;
  int rc = step_direct(b);
  cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
  b->graph_launches = b->launches - launches;
  b->launches = launches;
  if (rc || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return HWENO_ECUDA;
  }
  ce = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return HWENO_ECUDA;
  }
  b->graph_ok = true;
  return HWENO_OK;
}

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;  // batch signature -> (tiles/item, blocks/SM)

std::string signature(const hweno_batch* b) {
  std::string s;
  for (const hweno_ctx& h : b->inst)
    s += std::to_string(h.dim) + ":" + std::to_string(h.nx) + "x" + std::to_string(h.ny) + ";";
  return s;
}

}  // namespace

extern "C" {

int hweno_batch_create(int n, const hweno_desc* descs, hweno_batch_t** out) {
  if (!out) return HWENO_EINVAL;
  *out = nullptr;
  if (n <= 0 || !descs) return HWENO_EINVAL;
  hweno_batch* b = new (std::nothrow) hweno_batch();
  if (!b) return HWENO_ENOMEM;
  b->n = n;
  b->inst.resize(n);
  b->state_off.resize(n);
  b->ws_off.resize(n);
  size_t soff = 0, woff = 0;
  for (int i = 0; i < n; ++i) {
    const hweno_desc& d = descs[i];
    if (d.system != HWENO_EULER) {
      delete b;
      return HWENO_EINVAL;
    }
    hweno_t* tmp = nullptr;
    int rc = hweno_create(d.dim, d.system, d.nx, d.ny, d.dx, d.dy, d.gamma, d.bc, &tmp);
    if (rc) {
      delete b;
      return rc;
    }
    hweno_ctx& h = b->inst[i];
    h = *tmp;
    hweno_destroy(tmp);
    b->state_off[i] = soff;
    soff += hweno_state_doubles(&h);
    b->ws_off[i] = woff;
    woff += layout_of(&h).total;
  }
  b->state_total = soff;
  b->ws_inst_total = woff;
  // device tables: instance descriptors, alpha slots, work items (worst case: one tile per item)
  size_t ncells = 0, nfaces = 0;
  for (const hweno_ctx& h : b->inst) {
    ncells += (h.nx * h.ny + hw::kThreads - 1) / hw::kThreads;
    nfaces += ((h.nx + 1) * h.ny + hw::kThreads - 1) / hw::kThreads;
    if (h.dim == 2) nfaces += ((h.ny + 1) * h.nx + hw::kThreads - 1) / hw::kThreads;
  }
  b->ws_tables = align_up(n * sizeof(hw::BatchInst)) + align_up((size_t)4 * 2 * n * 8) +
                 align_up(ncells * sizeof(int2)) + align_up(nfaces * sizeof(int4));
  b->ws_total = b->ws_inst_total + b->ws_tables;
  b->stream = nullptr;
  b->state = nullptr;
  b->ws = nullptr;
  b->tiles_per_item = 1;
  b->blocks_per_sm = 0;
  b->graph_ok = false;
  b->launches = 0;
  int dev = 0;
  cudaDeviceProp prop;
  b->num_sms = 0;
  b->max_blocks_per_sm = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
    b->num_sms = prop.multiProcessorCount;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hw::k_batch_stage, hw::kThreads, 0) == cudaSuccess)
    b->max_blocks_per_sm = occ;
  void (*kern[2][3])(hw::BatchArgs) = {{hw::k_batch_cells<1>, hw::k_batch_faces<1>, hw::k_batch_update<1>},
                                       {hw::k_batch_cells<2>, hw::k_batch_faces<2>, hw::k_batch_update<2>}};
  for (int d = 0; d < 2; ++d)
    for (int ph = 0; ph < 3; ++ph) {
      int o = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern[d][ph], hw::kThreads, 0) != cudaSuccess) o = 1;
      b->occ_phase[d][ph] = std::max(1, o);
    }
  cudaGetLastError();
  b->blocks_per_sm = b->max_blocks_per_sm;
  b->mode = 1;
  *out = b;
  return HWENO_OK;
}

int hweno_batch_set_stream(hweno_batch_t* b, void* s) {
  if (!b) return HWENO_EINVAL;
  drop_graph(b);
  b->stream = static_cast<cudaStream_t>(s);
  for (hweno_ctx& h : b->inst) h.stream = b->stream;
  return HWENO_OK;
}

size_t hweno_batch_state_doubles(const hweno_batch_t* b) { return b ? b->state_total : 0; }

size_t hweno_batch_state_offset(const hweno_batch_t* b, int i) {
  return (b && i >= 0 && i < b->n) ? b->state_off[i] : 0;
}

size_t hweno_batch_workspace_bytes(const hweno_batch_t* b) { return b ? b->ws_total : 0; }

int hweno_batch_bind(hweno_batch_t* b, double* state_dev, void* ws) {
  if (!b || !state_dev || !ws) return HWENO_EINVAL;
  if (((uintptr_t)state_dev & 15) || ((uintptr_t)ws & 255)) return HWENO_EINVAL;
  if (b->num_sms <= 0 || b->max_blocks_per_sm <= 0) return HWENO_ECUDA;
  drop_graph(b);
  b->state = state_dev;
  b->ws = static_cast<unsigned char*>(ws);
  unsigned char* tables = b->ws + b->ws_inst_total;
  b->d_inst = reinterpret_cast<hw::BatchInst*>(tables);
  tables += align_up(b->n * sizeof(hw::BatchInst));
  b->alpha = reinterpret_cast<unsigned long long*>(tables);
  tables += align_up((size_t)4 * 2 * b->n * 8);
  b->d_cells = reinterpret_cast<int2*>(tables);
  size_t ncells = 0;
  for (const hweno_ctx& h : b->inst) ncells += (h.nx * h.ny + hw::kThreads - 1) / hw::kThreads;
  tables += align_up(ncells * sizeof(int2));
  b->d_faces = reinterpret_cast<int4*>(tables);
  std::vector<hw::BatchInst> hi(b->n);
  for (int i = 0; i < b->n; ++i) {
    hweno_ctx& h = b->inst[i];
    h.stream = b->stream;
    int rc = hweno_bind(&h, b->state + b->state_off[i], b->ws + b->ws_off[i]);
    if (rc) return rc;
    // the batch keeps slot s of every instance contiguous: [slot][instance][direction]
    h.w.alpha = b->alpha + 2 * i;
    h.w.astride = 2 * b->n;
    hi[i].g = grid_of(&h);
    hi[i].w = h.w;
    hi[i].S = h.state;
    hi[i].dim = h.dim;
    hi[i].pad_ = 0;
  }
  if (cudaMemsetAsync(b->alpha, 0, (size_t)4 * 2 * b->n * 8, b->stream) != cudaSuccess) return HWENO_ECUDA;
  if (cudaMemcpyAsync(b->d_inst, hi.data(), hi.size() * sizeof(hw::BatchInst), cudaMemcpyHostToDevice, b->stream) !=
      cudaSuccess)
    return HWENO_ECUDA;
  return upload_items(b);
}

int hweno_batch_set_time(hweno_batch_t* b, double t_end) {
  if (!b) return HWENO_EINVAL;
  if (!b->ws) return HWENO_ESTATE;
  for (hweno_ctx& h : b->inst) {
    int rc = hweno_set_time(&h, 0.0, t_end);
    if (rc) return rc;
  }
  return HWENO_OK;
}

int hweno_batch_step(hweno_batch_t* b, int nsteps) {
  if (!b || nsteps < 0) return HWENO_EINVAL;
  if (!b->ws) return HWENO_ESTATE;
  if (!b->graph_ok && build_graph(b) != HWENO_OK) drop_graph(b);
  for (int s = 0; s < nsteps; ++s) {
    if (b->graph_ok) {
      if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess) return HWENO_ECUDA;
      b->launches += b->graph_launches;
    } else {
      int rc = step_direct(b);
      if (rc) return rc;
    }
  }
  return HWENO_OK;
}

int hweno_batch_step_plain(hweno_batch_t* b, int nsteps) {
  if (!b || nsteps < 0) return HWENO_EINVAL;
  if (!b->ws) return HWENO_ESTATE;
  static const double a_k[3] = {0.0, 0.75, 1.0 / 3.0};
  static const double b_k[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int s = 0; s < nsteps; ++s) {
    for (int st = 0; st < 3; ++st) {
      if (cudaMemsetAsync(b->alpha + (size_t)st * 2 * b->n, 0, 2 * b->n * sizeof(unsigned long long), b->stream) !=
          cudaSuccess)
        return HWENO_ECUDA;
      for (hweno_ctx& h : b->inst) {
        const Grid g = grid_of(&h);
        const Launchers& f = launchers(&h);
        f.cell(g, h.state, h.w, st, b->stream);
        f.face(g, h.state, h.w, st, b->stream);
        f.update(g, h.state, h.w, 0, st, a_k[st], b_k[st], 0.0, st, nullptr, nullptr, b->stream);
        b->launches += 3;
      }
      if (cudaGetLastError() != cudaSuccess) return HWENO_ECUDA;
    }
  }
  return HWENO_OK;
}

int hweno_batch_dts(hweno_batch_t* b, double* dt_host, double* t_host) {
  if (!b || !dt_host) return HWENO_EINVAL;
  if (!b->ws) return HWENO_ESTATE;
  int status = HWENO_OK;
  for (int i = 0; i < b->n; ++i) {
    double dt = 0.0, t = 0.0;
    int rc = hweno_last_dt(&b->inst[i], &dt, &t);
    if (rc == HWENO_ENONPHYS)
      status = rc;
    else if (rc)
      return rc;
    dt_host[i] = dt;
    if (t_host) t_host[i] = t;
  }
  return status;
}

int hweno_batch_tune(hweno_batch_t* b, double* backup_dev, int* tiles_per_item, int* blocks_per_sm) {
  if (!b || !backup_dev) return HWENO_EINVAL;
  if (!b->ws) return HWENO_ESTATE;
  const std::string sig = signature(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      b->tiles_per_item = it->second.first;
      b->mode = it->second.second == 0 ? 1 : 0;
      b->blocks_per_sm = it->second.second == 0 ? b->max_blocks_per_sm : it->second.second;
      drop_graph(b);
      int rc = upload_items(b);
      if (tiles_per_item) *tiles_per_item = b->tiles_per_item;
      if (blocks_per_sm) *blocks_per_sm = b->mode == 1 ? 0 : b->blocks_per_sm;
      return rc;
    }
  }
  // time one step of every candidate on a copy of the state, then restore it
  const size_t bytes = b->state_total * 8;
  if (cudaMemcpyAsync(backup_dev, b->state, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
    return HWENO_ECUDA;
  std::vector<cudaEvent_t> ev(2);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return HWENO_ECUDA;
  float best = 1e30f;
  int best_t = 1, best_b = b->max_blocks_per_sm, best_m = 1;
  for (int tpi = 1; tpi <= kMaxTilesPerItem; tpi *= 2) {
    b->tiles_per_item = tpi;
    if (upload_items(b)) return HWENO_ECUDA;
    // mode 1 (phase launches at full occupancy), then mode 0 for each resident-block count
    for (int cand = 0; cand <= b->max_blocks_per_sm; ++cand) {
      b->mode = cand == 0 ? 1 : 0;
      b->blocks_per_sm = cand == 0 ? b->max_blocks_per_sm : cand;
      if (cudaMemcpyAsync(b->state, backup_dev, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
        return HWENO_ECUDA;
      cudaEventRecord(ev[0], b->stream);
      int rc = step_direct(b);
      cudaEventRecord(ev[1], b->stream);
      if (rc) return rc;
      if (cudaEventSynchronize(ev[1]) != cudaSuccess) return HWENO_ECUDA;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (ms < best) {
        best = ms;
        best_t = tpi;
        best_b = b->blocks_per_sm;
        best_m = b->mode;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (cudaMemcpyAsync(b->state, backup_dev, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
    return HWENO_ECUDA;
  for (hweno_ctx& h : b->inst) {
    int rc = hweno_set_time(&h, 0.0, 0.0);
    if (rc) return rc;
  }
  b->tiles_per_item = best_t;
  b->blocks_per_sm = best_b;
  b->mode = best_m;
  drop_graph(b);
  int rc = upload_items(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[sig] = {best_t, best_m == 1 ? 0 : best_b};
  }
  if (tiles_per_item) *tiles_per_item = best_t;
  if (blocks_per_sm) *blocks_per_sm = best_m == 1 ? 0 : best_b;
  return rc;
}

long long hweno_batch_launch_count(const hweno_batch_t* b) { return b ? b->launches : -1; }

void hweno_batch_destroy(hweno_batch_t* b) {
  if (!b) return;
  drop_graph(b);
  delete b;
}

}  // extern "C"
