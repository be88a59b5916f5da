// Batched stepping of many independent lattices (declared in include/lbm.h).
//
// All members share one device arena: for member m two population copies (the layout of a
// single lattice) at arena + off[m], then the member table, the physics table, the work list
// and the per-member non-finite flags.  One launch of k_step_batch per time step covers every
// member: a grid of resident CTAs deals out the work list, whose items are tiles of roughly equal
// node count, largest first.  Runs of kGraphSteps steps are captured once in a CUDA graph and
// replayed.  The autotuner times candidate tiles by relaunching the step with the same parity
// (which only rewrites the spare copies), so tuning leaves the state unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbmch;

namespace {

constexpr int kGraphSteps = 16;  // even: a replay returns to the parity it started from
constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Candidate tiles of the batch kernel and work-item sizes (nodes per item).
const int kTiles[][2] = {{32, 4}, {64, 2}, {64, 4}, {128, 1}, {128, 2}, {256, 1}};
const int kTargets[] = {2048, 4096, 8192, 16384};
constexpr int kMinTarget = 2048;

// Columns a CTA of the tile covers: bx, or 2 bx for the paired 16-bit tile (two nodes per thread).
int tile_cols(const StepTile& t) { return t.pair ? 2 * t.bx : t.bx; }

int item_rows(const HostGeometry& g, int cols, int by, int target) {
  const int w = std::min(cols, g.nx);
  int rows = std::max(by, target / w);
  rows = (rows + by - 1) / by * by;
  return std::min(rows, (g.ny + by - 1) / by * by);
}

// Upper bound on the work list length over every candidate.
size_t max_items(const std::vector<HostGeometry>& geo) {
  size_t worst = 0;
  for (auto& t : kTiles) {
    size_t n = 0;
    for (auto& g : geo) {
      const int rows = item_rows(g, t[0], t[1], kMinTarget);
      n += (size_t)((g.nx + t[0] - 1) / t[0]) * ((g.ny + rows - 1) / rows);
    }
    worst = std::max(worst, n);
  }
  size_t n = 0;  // the paired tile: 256 columns
  for (auto& g : geo) {
    const int rows = item_rows(g, 256, 1, kMinTarget);
    n += (size_t)((g.nx + 255) / 256) * ((g.ny + rows - 1) / rows);
  }
  return std::max(worst, n);
}

struct Layout {
  std::vector<size_t> off, copy;
  size_t members_off, phys_off, items_off, flags_off, tcount_off, total;
  size_t nitems_max;
};

Layout layout(int prec, const std::vector<HostGeometry>& geo) {
  Layout L;
  size_t o = 0;
  for (auto& g : geo) {
    const size_t cb = copy_bytes(prec, g);
    L.off.push_back(o);
    L.copy.push_back(cb);
    o += 2 * cb;
  }
  const size_t count = geo.size();
  L.members_off = o;
  o = align_up(o + sizeof(BatchMember) * count);
  L.phys_off = o;
  o = align_up(o + phys_bytes(prec) * count);
  L.nitems_max = max_items(geo);
  L.items_off = o;
  o = align_up(o + sizeof(BatchItem) * L.nitems_max);
  L.flags_off = o;
  o = align_up(o + sizeof(int) * count);
  L.tcount_off = o;  // the time step in two parity slots (see launch_step_batch)
  o = align_up(o + 2 * sizeof(long long));
  L.total = o;
  return L;
}

thread_local char g_batch_err[512] = "";

// Winning (tile, target) per batch signature, shared by every batch in the process.
std::mutex g_cache_mutex;
std::map<std::string, std::pair<StepTile, int>> g_cache;

}  // namespace

struct lbm_batch {
  int count, prec, device, sms;
  std::vector<lbm_params> p;
  std::vector<HostGeometry> geo;
  std::vector<HostPhys> phys;
  Layout L;
  char* arena;
  bool owns;
  cudaStream_t stream;
  bool own_stream;
  StepTile tile;
  int target;
  int nitems;
  int grid;
  int parity;
  long long t;
  cudaGraphExec_t graph;
  bool graph_ok;
  char err[512];
};

namespace {

int fail(lbm_batch* b, int code, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  return code;
}

std::string signature(const lbm_batch* b) {
  std::vector<std::tuple<int, int, int>> sizes;  // nx, ny, walls: the tiles that can serve a member
  for (auto& g : b->geo) sizes.emplace_back(g.nx, g.ny, g.walls);
  std::sort(sizes.begin(), sizes.end());
  std::string s = "p" + std::to_string(b->prec) + "/sm" + std::to_string(b->sms) + "/";
  for (auto& z : sizes)
    s += std::to_string(std::get<0>(z)) + "x" + std::to_string(std::get<1>(z)) + (std::get<2>(z) ? "w," : ",");
  return s;
}

// Rebuild and upload the work list for a tile and item size; invalidates the graph.
cudaError_t build_items(lbm_batch* b, const StepTile& t, int target) {
  std::vector<BatchItem> items;
  const int cols = tile_cols(t);
  for (int m = 0; m < b->count; ++m) {
    const HostGeometry& g = b->geo[m];
    const int rows = item_rows(g, cols, t.by, target);
    for (int y0 = 0; y0 < g.ny; y0 += rows)
      for (int x0 = 0; x0 < g.nx; x0 += cols) items.push_back(BatchItem{m, x0, y0, rows});
  }
  if (items.size() > b->L.nitems_max) return cudaErrorInvalidValue;
  auto nodes = [&](const BatchItem& w) {
    const HostGeometry& g = b->geo[w.member];
    return (long long)std::min(cols, g.nx - w.x0) * std::min(w.rows, g.ny - w.y0);
  };
  std::stable_sort(items.begin(), items.end(),
                   [&](const BatchItem& a, const BatchItem& c) { return nodes(a) > nodes(c); });
  cudaError_t e = cudaMemcpyAsync(b->arena + b->L.items_off, items.data(), sizeof(BatchItem) * items.size(),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return e;
  b->tile = t;
  b->target = target;
  b->nitems = (int)items.size();
  b->grid = std::max(1, std::min(b->nitems, b->sms * batch_blocks_per_sm(b->prec, t)));
  if (b->graph_ok) {
    cudaGraphExecDestroy(b->graph);
    b->graph_ok = false;
  }
  return cudaSuccess;
}

// Every member's population buffer under 4 GiB: the step kernel forms plane offsets in 32 bits.
bool members_fit_32(const lbm_batch* b) {
  for (const HostGeometry& g : b->geo)
    if (pop_buffer_bytes(b->prec, g.plane) >= (size_t(1) << 32)) return false;
  return true;
}

// The paired 16-bit tile serves batches whose members are all periodic 16-bit lattices with even
// nx and buffers under 4 GiB.
bool pair_ok(const lbm_batch* b) {
  if (b->prec != 2 && b->prec != 3) return false;
  for (const HostGeometry& g : b->geo)
    if (g.walls || g.nx % 2) return false;
  return members_fit_32(b);
}

cudaError_t launch_one(lbm_batch* b, int parity) {
  return launch_step_batch(b->prec, b->tile, (const BatchItem*)(b->arena + b->L.items_off), b->nitems,
                           (const BatchMember*)(b->arena + b->L.members_off), b->arena + b->L.phys_off, parity,
                           (int*)(b->arena + b->L.flags_off), (long long*)(b->arena + b->L.tcount_off), b->grid,
                           members_fit_32(b), b->stream);
}

cudaError_t build_graph(lbm_batch* b) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < kGraphSteps && le == cudaSuccess; ++s) le = launch_one(b, s & 1);
  e = cudaStreamEndCapture(b->stream, &g);
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e == cudaSuccess) b->graph_ok = true;
  return e;
}

char* state_of(lbm_batch* b, int m) { return b->arena + b->L.off[m] + (size_t)b->parity * b->L.copy[m]; }
char* spare_of(lbm_batch* b, int m) { return b->arena + b->L.off[m] + (size_t)(1 - b->parity) * b->L.copy[m]; }

}  // namespace

extern "C" {

int lbm_batch_state_bytes(const lbm_params* params, int count, size_t* bytes) {
  if (!params || count < 1 || !bytes) return fail(nullptr, LBM_ERR_PARAM, "lbm_batch_state_bytes: bad arguments");
  std::vector<HostGeometry> geo(count);
  for (int m = 0; m < count; ++m) {
    HostPhys ph;
    const char* msg = validate_params(&params[m], &geo[m], &ph);
    if (msg) return fail(nullptr, LBM_ERR_PARAM, "lbm_batch_state_bytes: member %d: %s", m, msg);
    if (params[m].prec != params[0].prec)
      return fail(nullptr, LBM_ERR_PARAM, "lbm_batch_state_bytes: all members need the same precision");
  }
  *bytes = layout(params[0].prec, geo).total;
  return LBM_OK;
}

int lbm_batch_init(const lbm_params* params, int count, const double* const* phi0, void* device_buffer,
                   size_t buffer_bytes, void* stream, lbm_batch** out) {
  g_batch_err[0] = 0;
  if (!out) return fail(nullptr, LBM_ERR_PARAM, "lbm_batch_init: out is NULL");
  *out = nullptr;
  if (!params || count < 1 || !phi0) return fail(nullptr, LBM_ERR_PARAM, "lbm_batch_init: bad arguments");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return fail(nullptr, LBM_ERR_OOM, "lbm_batch_init: host allocation failed");
  b->count = count;
  b->prec = params[0].prec;
  b->p.assign(params, params + count);
  b->geo.resize(count);
  b->phys.resize(count);
  for (int m = 0; m < count; ++m) {
    const char* msg = validate_params(&params[m], &b->geo[m], &b->phys[m]);
    if (!msg && params[m].prec != b->prec) msg = "all members need the same precision";
    if (!msg && !phi0[m]) msg = "phi0 is NULL";
    if (msg) {
      fail(nullptr, LBM_ERR_PARAM, "lbm_batch_init: member %d: %s", m, msg);
      delete b;
      return LBM_ERR_PARAM;
    }
  }
  b->L = layout(b->prec, b->geo);
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (b->sms <= 0) b->sms = 152;
  if (device_buffer) {
    if (((uintptr_t)device_buffer % kAlign) != 0 || buffer_bytes < b->L.total) {
      fail(nullptr, device_buffer && buffer_bytes < b->L.total ? LBM_ERR_OOM : LBM_ERR_PARAM,
           "lbm_batch_init: device buffer must be 256-byte aligned and hold %zu bytes", b->L.total);
      const int code = buffer_bytes < b->L.total ? LBM_ERR_OOM : LBM_ERR_PARAM;
      delete b;
      return code;
    }
    b->arena = (char*)device_buffer;
    b->owns = false;
  } else {
    if (cudaMalloc((void**)&b->arena, b->L.total) != cudaSuccess) {
      cudaGetLastError();
      fail(nullptr, LBM_ERR_OOM, "lbm_batch_init: cudaMalloc(%zu) failed", b->L.total);
      delete b;
      return LBM_ERR_OOM;
    }
    b->owns = true;
  }
  b->own_stream = stream == nullptr;  // graphs cannot be captured on the legacy default stream
  if (b->own_stream) cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  else b->stream = (cudaStream_t)stream;
  b->parity = 0;
  b->t = 0;
  b->graph_ok = false;
  b->err[0] = 0;

  cudaError_t e = cudaSuccess;
  std::vector<BatchMember> mem(count);
  for (int m = 0; m < count; ++m) {
    const HostGeometry& g = b->geo[m];
    mem[m] = BatchMember{g.nx, g.ny, g.pitch, g.walls, g.plane, b->arena + b->L.off[m],
                         b->arena + b->L.off[m] + b->L.copy[m]};
    // Initial state: stage [phi | 0 | 0 | 1] in copy 1, equilibria + one collision into copy 0.
    const long long N = (long long)g.nx * g.ny;
    double* stage = (double*)mem[m].buf1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage, phi0[m], sizeof(double) * N, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(stage + N, 0, sizeof(double) * 2 * N, b->stream);
    if (e == cudaSuccess) e = launch_fill(stage + 3 * N, N, 1.0, b->stream);
    if (e == cudaSuccess) e = launch_init(b->prec, g, b->phys[m], stage, mem[m].buf0, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // phi0[m] may be pageable
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->arena + b->L.members_off, mem.data(), sizeof(BatchMember) * count,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = upload_phys(b->prec, b->phys.data(), count, b->arena + b->L.phys_off, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->arena + b->L.flags_off, 0, sizeof(int) * count, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->arena + b->L.tcount_off, 0, 2 * sizeof(long long), b->stream);
  if (e == cudaSuccess) {
    // Default: the paired 16-bit tile where it can serve the batch (periodic 16-bit sweep of 132
    // members 64^2..512^2 on GB300: 40.2k MLUPS against 34.8k for the best one-node tile), else
    // the one-node 64 x 4 tile; a cached autotune winner for the same member sizes overrides both.
    StepTile t{64, 4, 0, 0, 1};
    if (pair_ok(b)) {
      t = StepTile{128, 1, 0, 0, 1};
      t.pair = 1;
    }
    int target = 4096;
    {
      std::lock_guard<std::mutex> lock(g_cache_mutex);
      auto it = g_cache.find(signature(b));
      if (it != g_cache.end() && (!it->second.first.pair || pair_ok(b))) {
        t = it->second.first;
        target = it->second.second;
      }
    }
    e = build_items(b, t, target);
  }
  if (e != cudaSuccess) {
    fail(nullptr, LBM_ERR_CUDA, "lbm_batch_init: %s", cudaGetErrorString(e));
    lbm_batch_free(b);
    return LBM_ERR_CUDA;
  }
  *out = b;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
  if (!b) return LBM_ERR_PARAM;
  if (n < 0) return fail(b, LBM_ERR_PARAM, "lbm_batch_step: n must be >= 0");
  cudaError_t e = cudaSuccess;
  while (n > 0 && e == cudaSuccess) {
    if (b->parity == 0 && n >= kGraphSteps) {
      if (!b->graph_ok) e = build_graph(b);
      if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
      if (e == cudaSuccess) {
        n -= kGraphSteps;
        b->t += kGraphSteps;
      }
    } else {
      e = launch_one(b, b->parity);
      if (e == cudaSuccess) {
        b->parity ^= 1;
        --n;
        ++b->t;
      }
    }
  }
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_step: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_fields(lbm_batch* b, int member, double* rho, double* ux, double* uy, double* phi) {
  if (!b || member < 0 || member >= b->count) return fail(b, LBM_ERR_PARAM, "lbm_batch_fields: bad member");
  const HostGeometry& g = b->geo[member];
  const long long N = (long long)g.nx * g.ny;
  double* stage = (double*)spare_of(b, member);
  cudaError_t e = launch_fields(b->prec, g, b->phys[member], state_of(b, member), stage, b->stream);
  double* outs[4] = {rho, ux, uy, phi};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    if (outs[k]) e = cudaMemcpyAsync(outs[k], stage + k * N, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_fields: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_set_state(lbm_batch* b, int member, const float* state) {
  if (!b || member < 0 || member >= b->count || !state)
    return fail(b, LBM_ERR_PARAM, "lbm_batch_set_state: bad member or NULL state");
  if ((uintptr_t)state % 4 != 0) return fail(b, LBM_ERR_PARAM, "lbm_batch_set_state: state must be 4-byte aligned");
  const HostGeometry& g = b->geo[member];
  const long long N = (long long)g.nx * g.ny;
  double* stage = (double*)spare_of(b, member);
  cudaError_t e = launch_state_to_fields(state, N, stage, b->stream);
  if (e == cudaSuccess) e = launch_init(b->prec, g, b->phys[member], stage, state_of(b, member), b->stream);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_set_state: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_get_state(lbm_batch* b, int member, float* state) {
  if (!b || member < 0 || member >= b->count || !state)
    return fail(b, LBM_ERR_PARAM, "lbm_batch_get_state: bad member or NULL state");
  if ((uintptr_t)state % 4 != 0) return fail(b, LBM_ERR_PARAM, "lbm_batch_get_state: state must be 4-byte aligned");
  const HostGeometry& g = b->geo[member];
  const long long N = (long long)g.nx * g.ny;
  double* stage = (double*)spare_of(b, member);
  cudaError_t e = launch_fields(b->prec, g, b->phys[member], state_of(b, member), stage, b->stream);
  if (e == cudaSuccess) e = launch_fields_to_state(stage, N, state, b->stream);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_get_state: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch* b, int member, double* f, double* g) {
  if (!b || member < 0 || member >= b->count) return fail(b, LBM_ERR_PARAM, "lbm_batch_get_populations: bad member");
  const HostGeometry& geo = b->geo[member];
  const long long N = (long long)geo.nx * geo.ny;
  double* stage = (double*)spare_of(b, member);
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < 18 && e == cudaSuccess; ++q) {
    double* dst = q < 9 ? (f ? f + q * N : nullptr) : (g ? g + (q - 9) * N : nullptr);
    if (!dst) continue;
    e = launch_plane_get(b->prec, geo, state_of(b, member), q, stage, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, stage, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  }
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_get_populations: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_check(lbm_batch* b, int* nonfinite) {
  if (!b) return LBM_ERR_PARAM;
  std::vector<int> flags(b->count, 0);
  cudaError_t e = cudaMemcpyAsync(flags.data(), b->arena + b->L.flags_off, sizeof(int) * b->count,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_check: %s", cudaGetErrorString(e));
  int bad = 0;
  for (int m = 0; m < b->count; ++m) {
    if (nonfinite) nonfinite[m] = flags[m] != 0;
    bad += flags[m] != 0;
  }
  if (bad) {
    cudaMemsetAsync(b->arena + b->L.flags_off, 0, sizeof(int) * b->count, b->stream);
    cudaStreamSynchronize(b->stream);
    return fail(b, LBM_ERR_NONFINITE, "%d member(s) produced a non-finite rho or phi", bad);
  }
  return LBM_OK;
}

int lbm_batch_set_tile(lbm_batch* b, int bx, int by, int target_nodes) {
  if (!b) return LBM_ERR_PARAM;
  bool known = false;
  for (auto& t : kTiles) known |= (t[0] == bx && t[1] == by);
  if (!known || target_nodes < kMinTarget)
    return fail(b, LBM_ERR_PARAM, "lbm_batch_set_tile: tile %dx%d / %d nodes per item not available", bx, by,
                target_nodes);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = build_items(b, StepTile{bx, by, 0, 0, 1}, target_nodes);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_set_tile: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_set_kernel(lbm_batch* b, int variant, int target_nodes) {
  if (!b) return LBM_ERR_PARAM;
  if ((variant != LBM_KERNEL_GENERIC && variant != LBM_KERNEL_PAIR) || target_nodes < kMinTarget)
    return fail(b, LBM_ERR_PARAM, "lbm_batch_set_kernel: variant %d / %d nodes per item not available", variant,
                target_nodes);
  StepTile t{64, 4, 0, 0, 1};
  if (variant == LBM_KERNEL_PAIR) {
    if (!pair_ok(b))
      return fail(b, LBM_ERR_PARAM,
                  "lbm_batch_set_kernel: the paired kernel needs 16-bit members, all periodic with even nx");
    t = StepTile{128, 1, 0, 0, 1};
    t.pair = 1;
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = build_items(b, t, target_nodes);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_set_kernel: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_batch_get_kernel(const lbm_batch* b, int* variant) {
  if (!b) return LBM_ERR_PARAM;
  if (variant) *variant = b->tile.pair ? LBM_KERNEL_PAIR : LBM_KERNEL_GENERIC;
  return LBM_OK;
}

int lbm_batch_get_tile(const lbm_batch* b, int* bx, int* by, int* target_nodes, int* items, int* grid) {
  if (!b) return LBM_ERR_PARAM;
  if (bx) *bx = b->tile.bx;
  if (by) *by = b->tile.by;
  if (target_nodes) *target_nodes = b->target;
  if (items) *items = b->nitems;
  if (grid) *grid = b->grid;
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int trial_steps, double* best_ms) {
  if (!b) return LBM_ERR_PARAM;
  if (trial_steps < 1) return fail(b, LBM_ERR_PARAM, "lbm_batch_autotune: trial_steps must be >= 1");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  StepTile best_t = b->tile;
  int best_target = b->target;
  cudaError_t e = cudaSuccess;
  std::vector<StepTile> cands;
  for (auto& tt : kTiles) cands.push_back(StepTile{tt[0], tt[1], 0, 0, 1});
  if (pair_ok(b)) {
    StepTile t{128, 1, 0, 0, 1};
    t.pair = 1;
    cands.push_back(t);
  }
  for (const StepTile& t : cands) {
    for (int target : kTargets) {
      e = build_items(b, t, target);
      if (e != cudaSuccess) break;
      // Same parity every launch: each rewrites the spare copies from the unchanged state.
      for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_one(b, b->parity);
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int s = 0; s < trial_steps && e == cudaSuccess; ++s) e = launch_one(b, b->parity);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      ms /= trial_steps;
      if (ms < best) {
        best = ms;
        best_t = t;
        best_target = target;
      }
    }
    if (e != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = build_items(b, best_t, best_target);
  if (e != cudaSuccess) return fail(b, LBM_ERR_CUDA, "lbm_batch_autotune: %s", cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    g_cache[signature(b)] = {best_t, best_target};
  }
  if (best_ms) *best_ms = best;
  return LBM_OK;
}

long long lbm_batch_time(const lbm_batch* b) { return b ? b->t : -1; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_batch_err; }

void lbm_batch_free(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  if (b->owns && b->arena) cudaFree(b->arena);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
