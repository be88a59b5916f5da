// C ABI of the solver (declarations and contracts in include/lbm.h).
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbmch;

struct lbm_lattice {
  lbm_params p;
  HostGeometry geo;
  HostPhys phys;
  StepTile tile;
  cudaStream_t stream;
  int device;
  char* buf;        // [buffer 0 | buffer 1 | status block]
  size_t pop_bytes; // bytes of one population buffer (256-aligned)
  bool owns;
  int cur;          // which buffer holds the state
  int* flag;        // device: non-finite flag
  double* out4;     // device: reduction result
  long long t;
  char err[512];
};

namespace {

thread_local char g_init_err[512] = "";

// Autotuned tiles per (precision, nx, ny, boundary, SM count), shared by the process.
std::mutex g_tune_mutex;
std::map<std::string, StepTile> g_tune;

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kStatusBytes = 256;

void set_err(char* dst, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

int cuda_fail(lbm_lattice* h, const char* what, cudaError_t e) {
  set_err(h->err, "%s: %s", what, cudaGetErrorString(e));
  return LBM_ERR_CUDA;
}

std::string tune_key(const lbm_lattice* h, int sms) {
  return std::to_string(h->p.prec) + "/" + std::to_string(h->geo.nx) + "x" + std::to_string(h->geo.ny) + "/" +
         std::to_string(h->geo.walls) + "/" + std::to_string(sms);
}

char* state_buf(lbm_lattice* h) { return h->buf + (size_t)h->cur * h->pop_bytes; }

uint32_t step_key(uint32_t seed, long long t) { return sr_step_key(seed, t); }
char* other_buf(lbm_lattice* h) { return h->buf + (size_t)(1 - h->cur) * h->pop_bytes; }

}  // namespace

// Validates parameters and fills the derived geometry/physics.  Returns a message or NULL.
const char* lbmch::validate_params(const lbm_params* p, HostGeometry* g, HostPhys* ph) {
  if (!p) return "params is NULL";
  if (p->nx < 3 || p->ny < 3) return "nx and ny must be >= 3";
  if (p->prec < LBM_FP64 || p->prec > LBM_BF16S) return "prec must be an lbm_precision";
  if (p->bc != LBM_PERIODIC && p->bc != LBM_WALLS_Y) return "bc must be an lbm_bc";
  if (p->visc != LBM_OMEGA_LINEAR && p->visc != LBM_TAU_LINEAR) return "visc must be an lbm_visc_interp";
  if (p->k8_form != LBM_K8_PROJECTED && p->k8_form != LBM_K8_PRINTED) return "k8_form must be an lbm_k8_form";
  if (p->collision != LBM_COLLIDE_CM && p->collision != LBM_COLLIDE_BGK) return "collision must be an lbm_collision";
  if (p->force_mode != LBM_FORCE_UNIFORM && p->force_mode != LBM_FORCE_PHASE_L)
    return "force_mode must be an lbm_force_mode";
  if (p->rounding != LBM_ROUND_NEAREST && p->rounding != LBM_ROUND_STOCHASTIC)
    return "rounding must be an lbm_rounding";
  if (p->rounding == LBM_ROUND_STOCHASTIC && p->prec != LBM_FP16S && p->prec != LBM_BF16S)
    return "stochastic rounding needs 16-bit storage (FP16S or BF16S)";
  const double vals[] = {p->tau_l,  p->tau_g,      p->M,       p->Gamma,   p->gamma,   p->a,      p->omega3,
                         p->u_top, p->u_bottom, p->wet_bottom, p->wet_top, p->force_x, p->force_y};
  for (double v : vals)
    if (!std::isfinite(v)) return "parameters must be finite";
  if (!(p->tau_l > 0.5) || !(p->tau_g > 0.5)) return "tau_l and tau_g must exceed 1/2 (positive viscosity)";
  if (!(p->M > 0) || !(p->Gamma > 0)) return "M and Gamma must be positive";
  if (p->gamma < 0 || p->a < 0) return "gamma and a must be >= 0";
  if (!(p->omega3 > 0 && p->omega3 < 2)) return "omega3 must lie in (0, 2)";
  if (p->bc != LBM_WALLS_Y && (p->wet_bottom != 0 || p->wet_top != 0))
    return "wet_bottom and wet_top need walls (bc = LBM_WALLS_Y)";
  const long long pitch = ((long long)p->nx + 31) / 32 * 32;
  if (pitch * (long long)p->ny > INT_MAX) return "lattice too large: pitch * ny must fit in int32";
  g->nx = p->nx;
  g->ny = p->ny;
  g->pitch = (int)pitch;
  g->plane = pitch * p->ny;
  g->walls = p->bc == LBM_WALLS_Y;
  const double cs2 = 1.0 / 3.0;
  ph->tau_l = p->tau_l;
  ph->tau_g = p->tau_g;
  ph->omega_l = 1.0 / p->tau_l;
  ph->omega_g = 1.0 / p->tau_g;
  ph->omega3 = p->omega3;
  ph->omega_phi = 1.0 / (p->M / (p->Gamma * cs2) + 0.5);
  ph->gamma = p->gamma;
  ph->a = p->a;
  ph->Gamma = p->Gamma;
  ph->u_top = p->u_top;
  ph->u_bottom = p->u_bottom;
  ph->wet_bottom = g->walls ? p->wet_bottom : 0.0;
  ph->wet_top = g->walls ? p->wet_top : 0.0;
  ph->force_x = p->force_x;
  ph->force_y = p->force_y;
  ph->force_mode = p->force_mode;
  ph->visc = p->visc;
  ph->k8_printed = p->k8_form == LBM_K8_PRINTED;
  ph->bgk = p->collision == LBM_COLLIDE_BGK;
  ph->rounding = p->rounding;
  ph->seed = p->seed;
  ph->sr_key = 0;
  return nullptr;
}

size_t lbmch::copy_bytes(int prec, const HostGeometry& g) {
  size_t pb = align_up(pop_buffer_bytes(prec, g.plane));
  // The non-state buffer doubles as scratch for staging the fields (4 nx*ny FP64) and the
  // reduction partials; make sure it is large enough for both.
  const size_t need = align_up(sizeof(double) * 4 * (size_t)g.nx * g.ny) + reduce_partials_bytes();
  if (pb < need) pb = align_up(need);
  return pb;
}

namespace {

size_t total_bytes(int prec, const HostGeometry& g, size_t* pop_bytes) {
  const size_t pb = copy_bytes(prec, g);
  if (pop_bytes) *pop_bytes = pb;
  return 2 * pb + kStatusBytes;
}

}  // namespace

void lbmch::set_thread_error(const char* msg) { std::snprintf(g_init_err, sizeof(g_init_err), "%s", msg); }

extern "C" {

double lbm_wall_gradient(double theta, double a, double gamma) {
  if (!(gamma > 0) || !(a >= 0)) return std::nan("");
  const double pi = 3.14159265358979323846;
  const double s = std::sin(theta);
  const double c = std::cos(std::acos(s * s) / 3.0);
  const double mag = std::sqrt(2.0 * a / gamma * c * (1.0 - c));
  return theta < 0.5 * pi ? mag : (theta > 0.5 * pi ? -mag : 0.0);
}

void lbm_default_params(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tau_l = 0.8;
  p->tau_g = 0.8;
  p->M = 0.1;
  p->Gamma = 1.0;
  p->gamma = 0.04;
  p->a = 0.04;
  p->omega3 = 1.0;
  p->k8_form = LBM_K8_PROJECTED;
  p->visc = LBM_OMEGA_LINEAR;
  p->bc = LBM_PERIODIC;
  p->prec = LBM_FP32;
  p->collision = LBM_COLLIDE_CM;
}

int lbm_state_bytes(const lbm_params* p, size_t* bytes) {
  HostGeometry g;
  HostPhys ph;
  const char* m = validate_params(p, &g, &ph);
  if (m) {
    set_err(g_init_err, "lbm_state_bytes: %s", m);
    return LBM_ERR_PARAM;
  }
  if (!bytes) return LBM_ERR_PARAM;
  *bytes = total_bytes(p->prec, g, nullptr);
  return LBM_OK;
}

int lbm_init(const lbm_params* p, const double* phi0, const double* ux0, const double* uy0,
             const double* rho0, void* device_buffer, size_t buffer_bytes, void* stream,
             lbm_lattice** out) {
  g_init_err[0] = 0;
  if (!out) {
    set_err(g_init_err, "lbm_init: out is NULL");
    return LBM_ERR_PARAM;
  }
  *out = nullptr;
  HostGeometry g;
  HostPhys ph;
  const char* m = validate_params(p, &g, &ph);
  if (m) {
    set_err(g_init_err, "lbm_init: %s", m);
    return LBM_ERR_PARAM;
  }
  if (!phi0) {
    set_err(g_init_err, "lbm_init: phi0 is NULL");
    return LBM_ERR_PARAM;
  }
  const long long N = (long long)g.nx * g.ny;
  const double* ins[4] = {phi0, ux0, uy0, rho0};
  for (int k = 0; k < 4; ++k) {
    if (!ins[k]) continue;
    for (long long n = 0; n < N; ++n)
      if (!std::isfinite(ins[k][n])) {
        set_err(g_init_err, "lbm_init: non-finite initial field %d at node %lld", k, n);
        return LBM_ERR_PARAM;
      }
  }
  if (device_buffer && ((uintptr_t)device_buffer % kAlign) != 0) {
    set_err(g_init_err, "lbm_init: device_buffer must be %zu-byte aligned", kAlign);
    return LBM_ERR_PARAM;
  }
  size_t pop_bytes = 0;
  const size_t need = total_bytes(p->prec, g, &pop_bytes);
  if (device_buffer && buffer_bytes < need) {
    set_err(g_init_err, "lbm_init: device buffer of %zu bytes is smaller than the %zu needed", buffer_bytes, need);
    return LBM_ERR_OOM;
  }
  lbm_lattice* h = new (std::nothrow) lbm_lattice();
  if (!h) {
    set_err(g_init_err, "lbm_init: host allocation failed");
    return LBM_ERR_OOM;
  }
  h->p = *p;
  h->geo = g;
  h->phys = ph;
  h->stream = (cudaStream_t)stream;
  h->pop_bytes = pop_bytes;
  h->cur = 0;
  h->t = 0;
  h->err[0] = 0;
  cudaGetDevice(&h->device);
  if (device_buffer) {
    h->buf = (char*)device_buffer;
    h->owns = false;
  } else {
    cudaError_t e = cudaMalloc((void**)&h->buf, need);
    if (e != cudaSuccess) {
      set_err(g_init_err, "lbm_init: cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
      delete h;
      cudaGetLastError();
      return LBM_ERR_OOM;
    }
    h->owns = true;
  }
  h->flag = (int*)(h->buf + 2 * pop_bytes);
  h->out4 = (double*)(h->buf + 2 * pop_bytes + 64);
  h->tile = default_tile(p->prec, g, h->device);
  {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(tune_key(h, sms > 0 ? sms : 152));
    if (it != g_tune.end()) h->tile = it->second;
  }

  // Stage the initial fields [phi | ux | uy | rho] in buffer 1, build the state in buffer 0.
  double* stage = (double*)(h->buf + pop_bytes);
  cudaError_t e = cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
  const double defaults[4] = {0.0, 0.0, 0.0, 1.0};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
    if (ins[k]) {
      e = cudaMemcpyAsync(stage + k * N, ins[k], sizeof(double) * N, cudaMemcpyHostToDevice, h->stream);
    } else if (defaults[k] == 0.0) {
      e = cudaMemsetAsync(stage + k * N, 0, sizeof(double) * N, h->stream);
    } else {
      e = launch_fill(stage + k * N, N, defaults[k], h->stream);
    }
  }
  if (e == cudaSuccess) e = launch_init(p->prec, g, ph, stage, h->buf, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    set_err(g_init_err, "lbm_init: %s", cudaGetErrorString(e));
    if (h->owns) cudaFree(h->buf);
    delete h;
    return LBM_ERR_CUDA;
  }
  *out = h;
  return LBM_OK;
}

int lbm_step(lbm_lattice* h, int n) {
  if (!h) return LBM_ERR_PARAM;
  if (n < 0) {
    set_err(h->err, "lbm_step: n must be >= 0");
    return LBM_ERR_PARAM;
  }
  HostPhys ph = h->phys;
  for (int s = 0; s < n; ++s) {
    if (ph.rounding == LBM_ROUND_STOCHASTIC) ph.sr_key = step_key(ph.seed, h->t);
    cudaError_t e = launch_step(h->p.prec, h->geo, ph, h->tile, state_buf(h), other_buf(h), h->flag, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, "lbm_step launch", e);
    h->cur = 1 - h->cur;
    ++h->t;
  }
  return LBM_OK;
}

int lbm_check(lbm_lattice* h) {
  if (!h) return LBM_ERR_PARAM;
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, "lbm_check", e);
  if (flag) {
    cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
    if (flag & kFlagTimeout) {
      set_err(h->err, "a bounded wait of the staged kernel gave up before time step %lld; the state is "
                      "incomplete until lbm_set_populations restores one", h->t);
      return LBM_ERR_TIMEOUT;
    }
    set_err(h->err, "non-finite rho or phi produced before time step %lld", h->t);
    return LBM_ERR_NONFINITE;
  }
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_lattice* h, int probes) {
  if (!h) return LBM_ERR_PARAM;
  h->phys.wait_probes = probes < 0 ? -1 : probes;
  return LBM_OK;
}

int lbm_fields(lbm_lattice* h, double* rho, double* ux, double* uy, double* phi) {
  if (!h) return LBM_ERR_PARAM;
  const long long N = (long long)h->geo.nx * h->geo.ny;
  double* stage = (double*)other_buf(h);
  cudaError_t e = launch_fields(h->p.prec, h->geo, h->phys, state_buf(h), stage, h->stream);
  double* outs[4] = {rho, ux, uy, phi};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    if (outs[k]) e = cudaMemcpyAsync(outs[k], stage + k * N, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, "lbm_fields", e);
  return lbm_check(h);
}

int lbm_conservation(lbm_lattice* h, double* sum_phi, double* sum_rho, double* mom) {
  if (!h) return LBM_ERR_PARAM;
  double* partials = (double*)other_buf(h);
  double res[4] = {0, 0, 0, 0};
  cudaError_t e = launch_reduce(h->p.prec, h->geo, state_buf(h), partials, h->out4, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, h->out4, sizeof(res), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, "lbm_conservation", e);
  if (sum_phi) *sum_phi = res[0];
  if (sum_rho) *sum_rho = res[1];
  if (mom) {
    mom[0] = res[2];
    mom[1] = res[3];
  }
  return LBM_OK;
}

int lbm_get_populations(lbm_lattice* h, double* f, double* g) {
  if (!h) return LBM_ERR_PARAM;
  const long long N = (long long)h->geo.nx * h->geo.ny;
  double* stage = (double*)other_buf(h);
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 18 && e == cudaSuccess; ++p) {
    double* dst = p < 9 ? (f ? f + p * N : nullptr) : (g ? g + (p - 9) * N : nullptr);
    if (!dst) continue;
    e = launch_plane_get(h->p.prec, h->geo, state_buf(h), p, stage, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, stage, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, "lbm_get_populations", e);
  return LBM_OK;
}

int lbm_set_populations(lbm_lattice* h, const double* f, const double* g) {
  if (!h) return LBM_ERR_PARAM;
  if (!f || !g) {
    set_err(h->err, "lbm_set_populations: f and g are required");
    return LBM_ERR_PARAM;
  }
  const long long N = (long long)h->geo.nx * h->geo.ny;
  double* stage = (double*)other_buf(h);
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 18 && e == cudaSuccess; ++p) {
    const double* src = p < 9 ? f + p * N : g + (p - 9) * N;
    e = cudaMemcpyAsync(stage, src, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_plane_set(h->p.prec, h->geo, state_buf(h), p, stage, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, "lbm_set_populations", e);
  return LBM_OK;
}

int lbm_set_kernel(lbm_lattice* h, int variant, int bx, int by, int depth, int rows) {
  if (!h) return LBM_ERR_PARAM;
  if (variant == LBM_KERNEL_AUTO) {
    StepTile t = default_tile(h->p.prec, h->geo, h->device);
    if (rows > 0) t.rows = rows;
    h->tile = t;
    return LBM_OK;
  }
  if ((variant != LBM_KERNEL_GENERIC && variant != LBM_KERNEL_STAGED && variant != LBM_KERNEL_GENERIC_WIDE &&
       variant != LBM_KERNEL_PAIR && variant != LBM_KERNEL_PAIR_STAGED) ||
      rows < 0 || bx < 0 || by < 0 || depth < 0) {
    set_err(h->err, "lbm_set_kernel: invalid arguments");
    return LBM_ERR_PARAM;
  }
  StepTile t;
  t.staged = variant == LBM_KERNEL_STAGED;
  t.bx = bx ? bx : (t.staged ? 64 : 256);
  t.by = by ? by : (t.staged ? 4 : 1);
  t.depth = depth ? depth : 1;
  t.rows = 0;
  t.wide = variant == LBM_KERNEL_GENERIC_WIDE;
  t.pair = variant == LBM_KERNEL_PAIR || variant == LBM_KERNEL_PAIR_STAGED;
  if (t.pair) {
    t.bx = bx ? bx : 128;
    t.by = by ? by : 1;
  }
  const bool pair_staged = variant == LBM_KERNEL_PAIR_STAGED;
  if (pair_staged) t.staged = 1;
  // The one-node staged kernel stores from shared memory without the node index the rounding
  // stream needs; the staged paired kernel stores from registers and rounds either way.
  const bool ok = pair_staged ? t.bx == 128 && t.by == 1 && pair_tma_supported(h->p.prec, h->geo, t.depth)
                  : t.staged  ? staged_supported(h->p.prec, h->geo, t) && h->phys.rounding == LBM_ROUND_NEAREST
                  : t.pair    ? pair_supported(h->p.prec, h->geo, t.bx, t.by)
                              : tile_supported(h->p.prec, t.bx, t.by);
  if (!ok) {
    set_err(h->err, "lbm_set_kernel: no %s kernel for tile %dx%d depth %d on this lattice (nx = %d)",
            pair_staged ? "staged paired 16-bit" : t.staged ? "staged" : (t.pair ? "paired 16-bit" : "generic"),
            t.bx, t.by, t.depth, h->geo.nx);
    return LBM_ERR_PARAM;
  }
  if (rows > 0) {
    t.rows = rows;
  } else {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int per_sm = pair_staged ? pair_tma_blocks_per_sm(h->p.prec, t.depth)
                       : t.staged  ? staged_blocks_per_sm(h->p.prec, t)
                       : t.pair    ? pair_blocks_per_sm(h->p.prec, t, h->geo.walls != 0)
                                   : generic_blocks_per_sm(h->p.prec, t);
    t.rows = default_rows(h->geo, t, (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 1));
  }
  h->tile = t;
  return LBM_OK;
}

int lbm_get_kernel(const lbm_lattice* h, int* variant, int* bx, int* by, int* depth, int* rows) {
  if (!h) return LBM_ERR_PARAM;
  if (variant)
    *variant = h->tile.staged && h->tile.pair ? LBM_KERNEL_PAIR_STAGED
               : h->tile.staged ? LBM_KERNEL_STAGED
               : h->tile.pair ? LBM_KERNEL_PAIR
               : (h->tile.wide || !offsets_fit_32(h->p.prec, h->geo.plane)) ? LBM_KERNEL_GENERIC_WIDE
                                                                            : LBM_KERNEL_GENERIC;
  if (bx) *bx = h->tile.bx;
  if (by) *by = h->tile.by;
  if (depth) *depth = h->tile.depth;
  if (rows) *rows = h->tile.rows;
  return LBM_OK;
}

int lbm_autotune(lbm_lattice* h, int trial_steps, double* best_ms) {
  if (!h) return LBM_ERR_PARAM;
  if (trial_steps < 1) {
    set_err(h->err, "lbm_autotune: trial_steps must be >= 1");
    return LBM_ERR_PARAM;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (sms <= 0) sms = 152;
  std::vector<StepTile> cands;
  const int gtiles[][2] = {{32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 1}, {128, 2}, {256, 1}};
  for (auto& gt : gtiles) {
    StepTile t{gt[0], gt[1], 0, 0, 1};
    t.rows = rows_for_wave(h->geo, t, sms * generic_blocks_per_sm(h->p.prec, t));
    cands.push_back(t);
    for (int r : {32, 64, 128})
      if (r % t.by == 0 && r < t.rows) cands.push_back(StepTile{gt[0], gt[1], r, 0, 1});
  }
  const int stiles[][3] = {{64, 4, 1}, {64, 2, 1}, {128, 2, 1}};
  for (auto& st : stiles) {
    StepTile t{st[0], st[1], 0, 1, st[2]};
    if (!staged_supported(h->p.prec, h->geo, t) || h->phys.rounding != LBM_ROUND_NEAREST) continue;
    t.rows = rows_for_wave(h->geo, t, sms * staged_blocks_per_sm(h->p.prec, t));
    cands.push_back(t);
  }
  const int ptiles[][2] = {{64, 2}, {128, 1}};
  for (auto& pt : ptiles) {
    if (!pair_supported(h->p.prec, h->geo, pt[0], pt[1])) continue;
    StepTile t{pt[0], pt[1], 0, 0, 1};
    t.pair = 1;
    t.rows = default_rows(h->geo, t, sms * pair_blocks_per_sm(h->p.prec, t, h->geo.walls != 0));
    cands.push_back(t);
  }
  for (int d : {1, 2}) {
    if (!pair_tma_supported(h->p.prec, h->geo, d)) continue;
    StepTile t{128, 1, 0, 1, d};
    t.pair = 1;
    t.rows = default_rows(h->geo, t, sms * pair_tma_blocks_per_sm(h->p.prec, d));
    cands.push_back(t);
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  StepTile best_t = h->tile;
  cudaError_t e = cudaSuccess;
  for (const StepTile& t : cands) {
    // Relaunching from the same state only rewrites the spare copy: the state is unchanged.
    for (int w = 0; w < 2 && e == cudaSuccess; ++w)
      e = launch_step(h->p.prec, h->geo, h->phys, t, state_buf(h), other_buf(h), h->flag, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int s = 0; s < trial_steps && e == cudaSuccess; ++s)
      e = launch_step(h->p.prec, h->geo, h->phys, t, state_buf(h), other_buf(h), h->flag, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= trial_steps;
    if (ms < best) {
      best = ms;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(h, "lbm_autotune", e);
  h->tile = best_t;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[tune_key(h, sms)] = best_t;
  }
  if (best_ms) *best_ms = best;
  return LBM_OK;
}

long long lbm_time(const lbm_lattice* h) { return h ? h->t : -1; }

const char* lbm_last_error(const lbm_lattice* h) { return h ? h->err : g_init_err; }

void lbm_free(lbm_lattice* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->owns) cudaFree(h->buf);
  delete h;
}

}  // extern "C"
