// md_api.cu -- host side of the C ABI declared in include/md.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/md.h"
#include "md_internal.cuh"

using namespace mdk;

extern "C" void md_destroy(md_ctx* c);

struct ReplicaHost {
  int64_t n_vap = 0, n_wall = 0;
  int32_t n_pores = 0, n_groups = 1, n_bins = 0;
  std::vector<double> wall;  // caller order, 3*n_wall
};

struct md_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;       // captures the bodies of conditional graph nodes
  bool own_stream = false;
  Arrays a{};
  PotDev pot{};
  Tuning tun{};
  bool mixed = false;
  int n_reps = 0;
  std::vector<RepDev> reps;
  std::vector<ReplicaHost> rh;
  std::vector<void*> allocs;
  std::string err;
  int32_t* status_host = nullptr;   // pinned: [0] device status bits, [1] the state check's row,
                                    // [2] the state load's rebuild flag
  int32_t* bad_row = nullptr;       // device: lowest row a state load's check rejected
  cudaEvent_t status_event = nullptr;
  bool status_pending = false;
  int last_status_bits = 0;
  int64_t steps_done = 0;
  int64_t bytes_h2d = 0, bytes_d2h = 0;
  int use_graph = 1, steps_per_graph = 10;
  bool method_chosen = false;       // the caller set pair_method: the autotuner keeps it
  cudaGraphExec_t graph_exec = nullptr;
  int graph_steps = 0;
  size_t prof_total = 0, groups_total = 0, pores_total = 0;
  double *stage_x = nullptr, *stage_v = nullptr;  // caller-order xyz rows (3 n_total each)
};

namespace {

thread_local std::string g_create_error;

md_status fail(md_ctx* c, md_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CUDA_TRY(ctx, call)                                                            \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail((ctx), MD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
md_status dalloc(md_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MD_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                  cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  e = cudaMemsetAsync(q, 0, bytes, c->stream);
  if (e != cudaSuccess) return fail(c, MD_ECUDA, cudaGetErrorString(e));
  return MD_OK;
}

uint32_t hi_word(double v) {
  uint64_t b;
  std::memcpy(&b, &v, 8);
  return (uint32_t)(b >> 32);
}

double lj_u(double r2, double eps, double sigma) {
  double s2 = sigma * sigma / r2, s6 = s2 * s2 * s2;
  return 4.0 * eps * (s6 * s6 - s6);
}

md_status validate_potential(md_ctx* c, const md_potential* p) {
  if (!p) return fail(c, MD_EINVAL, "potential is NULL");
  for (double q : {p->eps, p->sigma, p->mass, p->rc, p->eps_w, p->sigma_w, p->rc_w, p->skin,
                   p->r_ads, p->bin_width, p->cell_size})
    if (!std::isfinite(q)) return fail(c, MD_EINVAL, "potential: a parameter is not finite");
  if (p->cell_size < 0 ||
      (p->cell_size > 0 && p->cell_size < std::max(p->rc, p->rc_w) + p->skin))
    return fail(c, MD_EINVAL, "cell_size must be 0 or at least max(rc, rc_w) + skin");
  if (!(p->eps >= 0 && p->sigma > 0 && p->mass > 0 && p->rc > 0 && p->eps_w >= 0 &&
        p->sigma_w > 0 && p->rc_w > 0 && p->skin >= 0 && p->bin_width > 0))
    return fail(c, MD_EINVAL,
                "potential: eps, eps_w >= 0; sigma, mass, rc, rc_w, bin_width > 0; skin >= 0");
  if (p->r_ads > p->rc_w) return fail(c, MD_EINVAL, "r_ads must not exceed rc_w");
  if (p->precision != MD_PREC_FP64 && p->precision != MD_PREC_MIXED &&
      p->precision != MD_PREC_DF64)
    return fail(c, MD_EINVAL, "unknown precision");
  if (p->max_neighbors < 0 || p->max_wall_neighbors < 0)
    return fail(c, MD_EINVAL, "negative list capacity");
  if ((p->max_neighbors > 0 ? p->max_neighbors : 160) +
          (p->max_wall_neighbors > 0 ? p->max_wall_neighbors : 224) > kMaxCap)
    return fail(c, MD_EINVAL, "max_neighbors + max_wall_neighbors must not exceed 1023");
  return MD_OK;
}

md_status validate_system(md_ctx* c, const md_system* s, int r, double rl) {
  const std::string who = "replica " + std::to_string(r) + ": ";
  for (double q : {s->Lx, s->Ly, s->Lz, s->dt, s->T0, s->tau_B, s->slab_half, s->lattice_a})
    if (!std::isfinite(q))
      return fail(c, MD_EINVAL, who + "box, dt, T0, tau_B, slab_half and lattice_a must be finite");
  if (!(s->Lx > 0 && s->Ly > 0 && s->Lz > 0 && s->dt > 0 && s->T0 >= 0 && s->slab_half >= 0))
    return fail(c, MD_EINVAL, who + "box, dt must be > 0; T0, slab_half >= 0");
  if (s->n_vapor < 0 || s->n_wall < 0 || s->n_pores < 0)
    return fail(c, MD_EINVAL, who + "negative count");
  if (s->n_vapor > 0 && (!s->x0 || !s->v0)) return fail(c, MD_EINVAL, who + "x0/v0 NULL");
  if (s->n_pores > 0 && !s->pores) return fail(c, MD_EINVAL, who + "pores NULL");
  if (s->thermostat_every < 0) return fail(c, MD_EINVAL, who + "thermostat_every < 0");
  if (s->thermostat_every > 0 && s->tau_B > 0 && s->tau_B < s->thermostat_every * s->dt)
    return fail(c, MD_EINVAL, who + "tau_B below thermostat_every*dt would over-correct");
  if (!(std::floor(s->Lx / rl) >= 3 && std::floor(s->Ly / rl) >= 3))
    return fail(c, MD_EINVAL,
                who + "box x/y must hold at least 3 cells of max(rc,rc_w)+skin (or cell_size)");
  if (std::floor(s->Lx / rl) > 1023 || std::floor(s->Ly / rl) > 1023 ||
      std::floor(s->Lz / rl) > 1023)
    return fail(c, MD_EINVAL, who + "more than 1023 cells along an axis");
  if (!s->wall_xyz && !(s->lattice_a > 0) && s->slab_half > 0)
    return fail(c, MD_EINVAL, who + "lattice_a must be > 0 to generate the wall");
  for (int q = 0; q < s->n_pores; ++q) {
    const md_pore& P = s->pores[q];
    if (P.kind < 1 || P.kind > 5) return fail(c, MD_EINVAL, who + "unknown pore kind");
    for (double u : {P.cx, P.cy, P.r0, P.r1, P.r_cavity, P.width})
      if (!std::isfinite(u)) return fail(c, MD_EINVAL, who + "pore parameters must be finite");
    if (P.kind == MD_PORE_CONE && !(s->slab_half > 0))
      return fail(c, MD_EINVAL, who + "a cone needs slab_half > 0");
    if (P.kind == MD_PORE_PRISM && !(P.r0 > 0 && P.r1 > 0))
      return fail(c, MD_EINVAL, who + "a prism needs half-sides r0, r1 > 0");
    if (s->wall_model == MD_WALL_HARD && P.kind != MD_PORE_PRISM && P.kind != MD_PORE_SLIT)
      return fail(c, MD_EINVAL, who + "hard walls need prism or slit pores (axis-aligned faces)");
  }
  if (s->wall_model != MD_WALL_ATOMS && s->wall_model != MD_WALL_HARD)
    return fail(c, MD_EINVAL, who + "unknown wall model");
  if (s->wall_model == MD_WALL_HARD && s->wall_xyz && s->n_wall > 0)
    return fail(c, MD_EINVAL, who + "hard walls take no wall atoms");
  if (s->dims != 0 && s->dims != 2 && s->dims != 3)
    return fail(c, MD_EINVAL, who + "dims must be 0 (3), 2 or 3");
  if (s->dims == 2) {
    if (s->wall_model != MD_WALL_HARD)
      return fail(c, MD_EINVAL, who + "a planar system needs hard walls");
    for (int q = 0; q < s->n_pores; ++q)
      if (s->pores[q].kind != MD_PORE_PRISM)
        return fail(c, MD_EINVAL, who + "a planar system needs prism pores");
    for (int64_t i = 0; i < s->n_vapor; ++i)
      if (s->x0[3 * i + 1] != 0.0 || s->v0[3 * i + 1] != 0.0)
        return fail(c, MD_EINVAL, who + "a planar system needs y = 0 and vy = 0 for molecule " +
                                      std::to_string(i));
  }
  const double hx = 0.5 * s->Lx, hy = 0.5 * s->Ly, hz = 0.5 * s->Lz;
  for (int64_t i = 0; i < s->n_vapor; ++i) {
    const double* x = s->x0 + 3 * i;
    if (!(x[0] >= -hx && x[0] < hx && x[1] >= -hy && x[1] < hy && x[2] >= -hz && x[2] <= hz))
      return fail(c, MD_EINVAL, who + "molecule " + std::to_string(i) + " outside the box");
    const double* v = s->v0 + 3 * i;
    if (!(std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2])))
      return fail(c, MD_EINVAL, who + "non-finite velocity");
  }
  for (int64_t i = 0; s->wall_xyz && i < s->n_wall; ++i) {
    const double* x = s->wall_xyz + 3 * i;
    if (!(x[0] >= -hx && x[0] < hx && x[1] >= -hy && x[1] < hy && x[2] >= -hz && x[2] <= hz))
      return fail(c, MD_EINVAL, who + "wall atom " + std::to_string(i) + " outside the box");
  }
  return MD_OK;
}

// volume of a pore's carved region inside the slab |z| < h (closed forms); for a planar system
// (dims 2) the area in the x-z plane
double pore_volume(const md_pore& q, double Lx, double h, int dims) {
  const double pi = 3.14159265358979323846;
  switch (q.kind) {
    case MD_PORE_CYLINDER: return pi * q.r0 * q.r0 * 2.0 * h;
    case MD_PORE_CONE: return pi / 3.0 * 2.0 * h * (q.r0 * q.r0 + q.r0 * q.r1 + q.r1 * q.r1);
    case MD_PORE_SLIT: return q.width * Lx * 2.0 * h;
    case MD_PORE_INKBOTTLE: {
      // neck cylinder plus the part of the cavity sphere outside it, within the slab
      double v = pi * q.r0 * q.r0 * 2.0 * h;
      const double a2 = q.r_cavity * q.r_cavity - q.r0 * q.r0;
      if (a2 > 0.0) {
        const double zt = std::min(std::sqrt(a2), h);
        v += 2.0 * pi * (a2 * zt - zt * zt * zt / 3.0);
      }
      return v;
    }
    case MD_PORE_PRISM: {
      const double depth = h - prism_floor(q.width, h) < 2.0 * h ? h - prism_floor(q.width, h)
                                                                   : 2.0 * h;
      return (dims == 2 ? 2.0 * q.r0 : 4.0 * q.r0 * q.r1) * depth;
    }
    default: return 0.0;
  }
}

double min_img(double d, double L) {
  if (d >= 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

// simple-cubic wall sites -L/2 + (i + 1/2) a in |z| < h, minus every pore's carved region
std::vector<double> generate_wall(const md_system* s) {
  std::vector<double> w;
  if (!(s->slab_half > 0)) return w;
  const double a = s->lattice_a;
  const int nx = (int)std::llround(s->Lx / a), ny = (int)std::llround(s->Ly / a),
            nz = (int)std::llround(s->Lz / a);
  for (int k = 0; k < nz; ++k) {
    const double z = -0.5 * s->Lz + (k + 0.5) * a;
    if (!(std::fabs(z) < s->slab_half)) continue;
    for (int j = 0; j < ny; ++j) {
      const double y = -0.5 * s->Ly + (j + 0.5) * a;
      for (int i = 0; i < nx; ++i) {
        const double x = -0.5 * s->Lx + (i + 0.5) * a;
        bool carved = false;
        for (int q = 0; q < s->n_pores && !carved; ++q) {
          const md_pore& P = s->pores[q];
          carved = in_pore(P.kind, P.r0, P.r1, P.r_cavity, P.width, min_img(x - P.cx, s->Lx),
                           min_img(y - P.cy, s->Ly), z, s->slab_half);
        }
        if (!carved) {
          w.push_back(x);
          w.push_back(y);
          w.push_back(z);
        }
      }
    }
  }
  return w;
}

int status_to_code(int bits) {
  if (bits & kStatusOverflow) return MD_EOVERFLOW;
  if (bits & kStatusUnstable) return MD_EUNSTABLE;
  if (bits & kStatusTimeout) return MD_ETIMEOUT;
  if (bits & kStatusBounds) return MD_EBOUNDS;
  return MD_OK;
}

md_status device_status(md_ctx* c) {
  if (c->last_status_bits) {
    md_status s = (md_status)status_to_code(c->last_status_bits);
    if (c->err.empty()) c->err = md_status_string(s);
    return s;
  }
  return MD_OK;
}

// the status word's copy to the host, enqueued
md_status enqueue_status(md_ctx* c) {
  CUDA_TRY(c, cudaMemcpyAsync(c->status_host, c->a.status, sizeof(int32_t),
                              cudaMemcpyDeviceToHost, c->stream));
  c->bytes_d2h += sizeof(int32_t);
  return MD_OK;
}

md_status status_after_sync(md_ctx* c);

md_status sync_status(md_ctx* c) {
  md_status e = enqueue_status(c);
  if (e != MD_OK) return e;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_after_sync(c);
}

// the status word copied by enqueue_status, once the stream has reached it
md_status status_after_sync(md_ctx* c) {
  c->status_pending = false;
  c->last_status_bits = *c->status_host;
  if (c->last_status_bits) {
    md_status s = (md_status)status_to_code(c->last_status_bits);
    c->err = std::string("device reported: ") + md_status_string(s);
    if (s == MD_EBOUNDS) {  // the checked build names the check that failed first
      int32_t line = 0;
      if (cudaMemcpy(&line, c->a.status + 1, sizeof(line), cudaMemcpyDeviceToHost) == cudaSuccess)
        c->err += " (md_kernels.cu line " + std::to_string(line) + ")";
      cudaGetLastError();
    }
    return s;
  }
  return MD_OK;
}

// what the first half-kick does besides Fig. 2: clear the forces for the FP64 atomic pair pass;
// refresh the FP32 cell-local offsets for the kernels that screen or compute with them
int integrate_flags(const md_ctx* c) {
  int f = 0;
  if (c->tun.atomic_acc || c->tun.cells) f |= kIntZeroForces;
  if (c->mixed || c->tun.tpp_fp64 >= 32 || c->tun.cells) f |= kIntLocalOffsets;
  if (c->tun.df64) f |= kIntLocalOffsets | kIntLocalOffsetsLo;
  return f;
}

// One step with plain launches: the rebuild kernels always launch and return at once when the
// device decides they have nothing to do. A thermostat step's scaling is paid by the next step's
// first kernel (or by launch_settle before a read).
void enqueue_step(md_ctx* c) {
  launch_integrate_first(c->a, c->pot, c->mixed, StepConds{}, integrate_flags(c), c->tun,
                         c->stream);
  if (!c->tun.all_pairs) launch_rebuild(c->a, c->pot, c->tun, c->mixed, c->stream);
  launch_forces(c->a, c->pot, c->mixed, false, true, c->tun, c->stream);
}

md_status rebuild_and_forces(md_ctx* c) {
  // the flag only needs to be nonzero: a memset, no copy from pageable host memory
  CUDA_TRY(c, cudaMemsetAsync(c->a.force_rebuild, 0x01, sizeof(int), c->stream));
  // every replica rebuilds (all-ones bytes: the largest displacement pattern)
  CUDA_TRY(c, cudaMemsetAsync(c->a.rep_disp2, 0xff, sizeof(unsigned long long) * (size_t)c->n_reps,
                              c->stream));
  launch_rebuild(c->a, c->pot, c->tun, c->mixed, c->stream);
  launch_forces(c->a, c->pot, c->mixed, false, false, c->tun, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  return sync_status(c);
}

void destroy_graph(md_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  c->graph_steps = 0;
}

// Append an IF node on `handle` to the graph being captured on c->stream and capture `body`
// (launches on the given stream) into its body graph.
template <typename Body>
cudaError_t add_conditional(md_ctx* c, cudaGraph_t g, cudaGraphConditionalHandle handle,
                            Body body) {
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, nullptr, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = handle;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  cudaGraph_t bg = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(c->aux, bg, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  body(c->aux);
  cudaGraph_t out = nullptr;
  return cudaStreamEndCapture(c->aux, &out);
}

// Capture `steps` MD steps as one graph. The rebuild chain sits in a conditional node whose
// condition the last block of k_integrate_first sets, so steps without a rebuild launch only the
// integrate and force kernels; the thermostat lives inside the integrate kernel.
md_status build_graph(md_ctx* c, int steps) {
  destroy_graph(c);
  if (!c->aux) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
  CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  for (int k = 0; k < steps && e == cudaSuccess; ++k) {
    StepConds sc;
    sc.use = 1;
    sc.has_rebuild = c->tun.all_pairs ? 0 : 1;
    if (sc.has_rebuild)
      e = cudaGraphConditionalHandleCreate(&sc.rebuild, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) break;
    launch_integrate_first(c->a, c->pot, c->mixed, sc, integrate_flags(c), c->tun, c->stream);
    if (sc.has_rebuild)
      e = add_conditional(c, g, sc.rebuild, [&](cudaStream_t s) {
        launch_rebuild(c->a, c->pot, c->tun, c->mixed, s);
      });
    if (e != cudaSuccess) break;
    launch_forces(c->a, c->pot, c->mixed, false, true, c->tun, c->stream);
  }
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->stream, &captured);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (captured) cudaGraphDestroy(captured);
    cudaGetLastError();
    return fail(c, MD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&c->graph_exec, captured, 0);
  cudaGraphDestroy(captured);
  if (e != cudaSuccess)
    return fail(c, MD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  c->graph_steps = steps;
  return MD_OK;
}

bool check_replica(md_ctx* c, int32_t r) { return c && r >= 0 && r < c->n_reps; }

md_status create_impl(const md_system* systems, int32_t n_reps, const md_potential* pot,
                      void* stream, md_ctx** out) {
  if (!out) return MD_EINVAL;
  *out = nullptr;
  md_ctx* c = new md_ctx();
  md_status st = MD_OK;
  auto bail = [&](md_status s) {
    g_create_error = c->err.empty() ? md_status_string(s) : c->err;
    md_destroy(c);
    return s;
  };
  // all argument checks come before the first CUDA call
  if (!systems || n_reps <= 0) return bail(fail(c, MD_EINVAL, "no systems"));
  if ((st = validate_potential(c, pot)) != MD_OK) return bail(st);
  const double rl = std::max(pot->rc, pot->rc_w) + pot->skin;
  const double cell = std::max(rl, pot->cell_size);  // cell side: at least the list radius
  for (int r = 0; r < n_reps; ++r)
    if ((st = validate_system(c, &systems[r], r, cell)) != MD_OK) return bail(st);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(c, MD_ECUDA, cudaGetErrorString(e)));
    c->own_stream = true;
  }
  {
    const cudaError_t e =
        configure_kernels(&c->tun.integrate_blocks_per_sm, &c->tun.small_blocks_per_sm);
    if (e != cudaSuccess) return bail(fail(c, MD_ECUDA, cudaGetErrorString(e)));
  }
  c->n_reps = n_reps;
  c->mixed = pot->precision == MD_PREC_MIXED;
  if (pot->precision == MD_PREC_DF64) {
    // an FP64 context whose pair terms run in double-float on the FP32 pipe: atomic reaction
    // forces by default, and the launch shape of an FP32-pipe kernel until the autotuner says
    // otherwise
    c->tun.df64 = 1;
    c->tun.atomic_acc = 1;
    c->tun.tpp_fp64 = 4;
    c->tun.force_blocks_per_sm_fp64 = 4;
  }

  // ---- potential constants
  PotDev& P = c->pot;
  const double s6 = std::pow(pot->sigma, 6), s12 = s6 * s6;
  const double w6 = std::pow(pot->sigma_w, 6), w12 = w6 * w6;
  P.rc2 = pot->rc * pot->rc;
  P.rcw2 = pot->rc_w * pot->rc_w;
  P.a12 = 48.0 * pot->eps * s12;
  P.b6 = 24.0 * pot->eps * s6;
  P.a12w = 48.0 * pot->eps_w * w12;
  P.b6w = 24.0 * pot->eps_w * w6;
  P.e12 = 4.0 * pot->eps * s12;
  P.e6 = 4.0 * pot->eps * s6;
  P.e12w = 4.0 * pot->eps_w * w12;
  P.e6w = 4.0 * pot->eps_w * w6;
  P.ushift = pot->shift_energy ? lj_u(P.rc2, pot->eps, pot->sigma) : 0.0;
  P.ushift_w = pot->shift_energy ? lj_u(P.rcw2, pot->eps_w, pot->sigma_w) : 0.0;
  P.mass = pot->mass;
  P.inv_mass = 1.0 / pot->mass;
  // (0.1 % early: the FP32 displacement errs by ~1e-6 of the skin, far inside that margin)
  P.half_skin2 = 0.25 * pot->skin * pot->skin * (1.0 - 1e-3);
  P.group_disp2 = 0.36 * P.half_skin2;  // 0.6 skin/2
  P.r_ads2 = pot->r_ads * pot->r_ads;
  P.rc2f = (float)P.rc2;
  P.rcw2f = (float)P.rcw2;
  P.rl2f = (float)((rl + 1e-4) * (rl + 1e-4));
  P.a12f = (float)P.a12;
  P.b6f = (float)P.b6;
  P.a12wf = (float)P.a12w;
  P.b6wf = (float)P.b6w;
  P.a12l = (float)(P.a12 - (double)P.a12f);
  P.b6l = (float)(P.b6 - (double)P.b6f);
  P.a12wl = (float)(P.a12w - (double)P.a12wf);
  P.b6wl = (float)(P.b6w - (double)P.b6wf);
  P.e12f = (float)P.e12;
  P.e6f = (float)P.e6;
  P.e12wf = (float)P.e12w;
  P.e6wf = (float)P.e6w;
  P.rc2f_lo = (float)(P.rc2 * (1.0 - 1e-5));
  P.rc2f_hi = (float)(P.rc2 * (1.0 + 1e-5));
  P.rcw2f_lo = (float)(P.rcw2 * (1.0 - 1e-5));
  P.rcw2f_hi = (float)(P.rcw2 * (1.0 + 1e-5));
  P.cap_v = pot->max_neighbors > 0 ? pot->max_neighbors : 160;
  P.cap = P.cap_v + (pot->max_wall_neighbors > 0 ? pot->max_wall_neighbors : 224);

  // ---- replicas, walls, cells
  c->reps.resize(n_reps);
  c->rh.resize(n_reps);
  std::vector<PoreDev> pores;
  std::vector<double> ctr;  // cell centres, per replica x then y then z
  long long n_tot = 0, nw_tot = 0, ncell_tot = 0, groups = 0, prof = 0;
  for (int r = 0; r < n_reps; ++r) {
    const md_system* s = &systems[r];
    ReplicaHost& H = c->rh[r];
    if (s->wall_model == MD_WALL_HARD)
      H.wall.clear();
    else if (s->wall_xyz)
      H.wall.assign(s->wall_xyz, s->wall_xyz + 3 * s->n_wall);
    else
      H.wall = generate_wall(s);
    H.n_vap = s->n_vapor;
    H.n_wall = (int64_t)(H.wall.size() / 3);
    H.n_pores = s->n_pores;
    H.n_groups = std::max(1, s->n_pores);
    H.n_bins = (int)std::ceil(s->Lz / pot->bin_width);
    RepDev& R = c->reps[r];
    R.Lx = s->Lx; R.Ly = s->Ly; R.Lz = s->Lz;
    R.hx = 0.5 * s->Lx; R.hy = 0.5 * s->Ly; R.hz = 0.5 * s->Lz;
    R.T0 = s->T0;
    R.dt = s->dt;
    R.n_th = s->thermostat_every;
    const double tau = s->tau_B > 0 ? s->tau_B : s->thermostat_every * s->dt;
    R.lam_coef = s->thermostat_every > 0 ? s->thermostat_every * s->dt / tau : 0.0;
    R.slab_half = s->slab_half;
    R.ncx = (int)std::floor(s->Lx / cell);
    R.ncy = (int)std::floor(s->Ly / cell);
    R.ncz = std::max(1, (int)std::floor(s->Lz / cell));
    R.lcx = s->Lx / R.ncx; R.lcy = s->Ly / R.ncy; R.lcz = s->Lz / R.ncz;
    R.ilcx = 1.0 / R.lcx; R.ilcy = 1.0 / R.lcy; R.ilcz = 1.0 / R.lcz;
    R.lcxf = (float)R.lcx; R.lcyf = (float)R.lcy; R.lczf = (float)R.lcz;
    R.lcx_lo = (float)(R.lcx - (double)R.lcxf);
    R.lcy_lo = (float)(R.lcy - (double)R.lcyf);
    R.lcz_lo = (float)(R.lcz - (double)R.lczf);
    R.hi_thr_x = hi_word(R.hx);
    R.hi_thr_y = hi_word(R.hy);
    R.bin_width = pot->bin_width;
    R.vap_off = (int32_t)n_tot;
    R.n_vap = (int32_t)H.n_vap;
    R.wall_off = (int32_t)nw_tot;
    R.n_wall = (int32_t)H.n_wall;
    R.cell_off = (int32_t)ncell_tot;
    R.pore_off = (int32_t)pores.size();
    R.n_pores = s->n_pores;
    R.group_off = (int32_t)groups;
    R.n_groups = H.n_groups;
    R.n_bins = H.n_bins;
    R.prof_off = (int32_t)prof;
    R.half_dt_m = 0.5 * s->dt * (1.0 / pot->mass);
    R.dt_m = s->dt * (1.0 / pot->mass);
    R.ctr_off = (int32_t)ctr.size();
    for (int k = 0; k < R.ncx; ++k) ctr.push_back(-R.hx + (k + 0.5) * R.lcx);
    for (int k = 0; k < R.ncy; ++k) ctr.push_back(-R.hy + (k + 0.5) * R.lcy);
    for (int k = 0; k < R.ncz; ++k) ctr.push_back(-R.hz + (k + 0.5) * R.lcz);
    R.dims = s->dims == 2 ? 2 : 3;
    R.hard = s->wall_model == MD_WALL_HARD ? 1 : 0;
    for (int q = 0; q < s->n_pores; ++q) {
      const md_pore& Q = s->pores[q];
      pores.push_back(PoreDev{Q.kind, Q.cx, Q.cy, Q.r0, Q.r1, Q.r_cavity, Q.width,
                              pore_volume(Q, s->Lx, s->slab_half, R.dims)});
    }
    n_tot += H.n_vap;
    nw_tot += H.n_wall;
    ncell_tot += (long long)R.ncx * R.ncy * R.ncz;
    groups += H.n_groups;
    prof += (long long)H.n_groups * H.n_bins;
  }
  if (n_tot + nw_tot > kMaxIndex)
    return bail(fail(c, MD_EINVAL, "more than 2^26 - 1 molecules plus wall atoms in one context"));
  if (ncell_tot > 4096LL * 4096LL) return bail(fail(c, MD_EINVAL, "too many cells"));
  if (!c->mixed && (unsigned long long)n_tot * (unsigned long long)c->pot.cap_v >= 0xffffffffull)
    return bail(fail(c, MD_EINVAL,
                     "FP64 pair buffer: molecules * max_neighbors must stay below 2^32"));
  c->prof_total = (size_t)prof;
  c->groups_total = (size_t)groups;
  c->pores_total = pores.size();

  // wall sorted by cell (stable): positions, FP32 offsets from the home-cell centre, CSR starts
  std::vector<int> wcell(nw_tot);
  std::vector<int32_t> wstart(ncell_tot + 1, 0);
  std::vector<dvec4> wpos(nw_tot);
  std::vector<float4> wlpos(nw_tot), wlpos_lo(nw_tot);
  std::vector<int32_t> cell_rep(ncell_tot);
  {
    long long k = 0;
    for (int r = 0; r < n_reps; ++r) {
      const RepDev& R = c->reps[r];
      for (long long q = 0; q < (long long)R.ncx * R.ncy * R.ncz; ++q) cell_rep[R.cell_off + q] = r;
      const std::vector<double>& W = c->rh[r].wall;
      for (int64_t i = 0; i < c->rh[r].n_wall; ++i, ++k) {
        int ix = cell_coord(W[3 * i], R.hx, R.lcx, R.ncx);
        int iy = cell_coord(W[3 * i + 1], R.hy, R.lcy, R.ncy);
        int iz = cell_coord(W[3 * i + 2], R.hz, R.lcz, R.ncz);
        wcell[k] = R.cell_off + (iz * R.ncy + iy) * R.ncx + ix;
        wstart[wcell[k] + 1] += 1;
      }
    }
    for (long long q = 0; q < ncell_tot; ++q) wstart[q + 1] += wstart[q];
    std::vector<int32_t> fill(wstart.begin(), wstart.end() - 1);
    k = 0;
    for (int r = 0; r < n_reps; ++r) {
      const RepDev& R = c->reps[r];
      const std::vector<double>& W = c->rh[r].wall;
      for (int64_t i = 0; i < c->rh[r].n_wall; ++i, ++k) {
        const int cell = wcell[k];
        const int dst = fill[cell]++;
        const double x = W[3 * i], y = W[3 * i + 1], z = W[3 * i + 2];
        wpos[dst] = make_dvec4(x, y, z, 0.0);
        const int local = cell - R.cell_off;
        const int ix = local % R.ncx, iy = (local / R.ncx) % R.ncy, iz = local / (R.ncx * R.ncy);
        const double cx = -R.hx + (ix + 0.5) * R.lcx, cy = -R.hy + (iy + 0.5) * R.lcy,
                     cz = -R.hz + (iz + 0.5) * R.lcz;
        const double lx = min_img(x - cx, R.Lx), ly = min_img(y - cy, R.Ly), lz = z - cz;
        wlpos[dst] = make_float4((float)lx, (float)ly, (float)lz, 0.f);
        wlpos_lo[dst] = make_float4((float)(lx - (double)wlpos[dst].x),
                                    (float)(ly - (double)wlpos[dst].y),
                                    (float)(lz - (double)wlpos[dst].z), 0.f);
      }
    }
  }

  // rows of cells (the cell method's work units) and, per cell, the wall atoms of its 27-cell
  // neighbourhood (x and y periodic, z bounded)
  std::vector<int32_t> row_cell, wnear(ncell_tot, 0);
  for (int r = 0; r < n_reps; ++r) {
    const RepDev& R = c->reps[r];
    for (int iz = 0; iz < R.ncz; ++iz)
      for (int iy = 0; iy < R.ncy; ++iy) {
        row_cell.push_back(R.cell_off + (iz * R.ncy + iy) * R.ncx);
        for (int ix = 0; ix < R.ncx; ++ix) {
          int32_t tot = 0;
          for (int dz = -1; dz <= 1; ++dz) {
            const int jz = iz + dz;
            if (jz < 0 || jz >= R.ncz) continue;
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int jy = (iy + dy + R.ncy) % R.ncy, jx = (ix + dx + R.ncx) % R.ncx;
                const int cn = R.cell_off + (jz * R.ncy + jy) * R.ncx + jx;
                tot += wstart[cn + 1] - wstart[cn];
              }
          }
          wnear[R.cell_off + (iz * R.ncy + iy) * R.ncx + ix] = tot;
        }
      }
  }
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
      c->tun.sm_count = sms;
    cudaGetLastError();
  }
  // ---- device memory
  Arrays& A = c->a;
  A.n_total = (int32_t)n_tot;
  A.n_wall_total = (int32_t)nw_tot;
  A.n_cells = (int32_t)ncell_tot;
  A.n_reps = n_reps;
  const size_t N = (size_t)n_tot;
#define ALLOC(ptr, cnt)                                 \
  if ((st = dalloc(c, &(ptr), (cnt))) != MD_OK) return bail(st)
  ALLOC(A.pos, N); ALLOC(A.vel, N); ALLOC(A.frc, N); ALLOC(A.lref, N);
  ALLOC(A.pos_alt, N); ALLOC(A.vel_alt, N); ALLOC(A.frc_alt, N);
  ALLOC(A.lpos, N); ALLOC(A.lpos_lo, N);
  ALLOC(c->stage_x, 3 * N); ALLOC(c->stage_v, 3 * N);
  ALLOC(A.home, N); ALLOC(A.id, N); ALLOC(A.rep, N); ALLOC(A.id_alt, N);
  ALLOC(A.cell_tmp, N); ALLOC(A.slot_tmp, N); ALLOC(A.perm_tmp, N);
  ALLOC(A.nbr, N * (size_t)P.cap);
  ALLOC(A.n_front, N); ALLOC(A.n_back, N); ALLOC(A.n_vh, N);
  ALLOC(A.order, N);
  ALLOC(A.hist, (size_t)kMaxCap + 2); ALLOC(A.hstart, (size_t)kMaxCap + 2);
  ALLOC(A.work, 1); ALLOC(A.work_done, 1);
  if (!c->mixed) {
    ALLOC(A.fwd, N * (size_t)P.cap_v);
    ALLOC(A.pairbuf, N * (size_t)P.cap_v + 1);
    ALLOC(A.fpart, N);
  }
  ALLOC(A.wpos, (size_t)nw_tot); ALLOC(A.wlpos, (size_t)nw_tot); ALLOC(A.wlpos_lo, (size_t)nw_tot);
  ALLOC(A.wstart, (size_t)ncell_tot + 1);
  ALLOC(A.vcount, (size_t)ncell_tot); ALLOC(A.vstart, (size_t)ncell_tot + 1);
  ALLOC(A.scan_tiles, 4096);
  RepDev* reps_d = nullptr;
  PoreDev* pores_d = nullptr;
  ALLOC(reps_d, (size_t)n_reps);
  ALLOC(pores_d, pores.size());
  A.reps = reps_d;
  A.pores = pores_d;
  int32_t* cell_rep_d = nullptr;
  ALLOC(cell_rep_d, (size_t)ncell_tot);
  A.cell_rep = cell_rep_d;
  if (n_tot <= kSmallMax) {  // the small-system method's absolute FP32 positions
    ALLOC(A.xf, N);
    ALLOC(A.xf_alt, N);
    float4* wxf_d = nullptr;
    ALLOC(wxf_d, (size_t)nw_tot);
    A.wxf = wxf_d;
  }
  int32_t *row_cell_d = nullptr, *wnear_d = nullptr;
  ALLOC(row_cell_d, row_cell.size());
  ALLOC(wnear_d, (size_t)ncell_tot);
  A.row_cell = row_cell_d;
  A.wnear = wnear_d;
  A.n_rows = (int32_t)row_cell.size();
  double* ctr_d = nullptr;
  ALLOC(ctr_d, ctr.size());
  A.cell_ctr = ctr_d;
  ALLOC(A.lambda, (size_t)n_reps);
  ALLOC(A.any_scale, 1);
  ALLOC(A.step, 1);
  ALLOC(A.force_rebuild, 1);
  ALLOC(A.kick_pending, 1); ALLOC(A.kick_done, 1); ALLOC(A.chain_done, 1);
  ALLOC(A.thermo_owed, 1); ALLOC(A.bar_arrive, 1); ALLOC(A.bar_release, 1);
  ALLOC(A.rep_disp2, (size_t)n_reps);
  ALLOC(A.act_cells, (size_t)ncell_tot); ALLOC(A.act_rep, (size_t)ncell_tot); ALLOC(A.act_home, (size_t)ncell_tot); ALLOC(A.n_act, 1);
  ALLOC(A.status, 2);
  ALLOC(A.n_rebuilds, 1);
  ALLOC(A.pair_count, 1);
  ALLOC(A.max_nb, 1);
  ALLOC(A.blk_done, 1);
  ALLOC(A.launch_count, 1);
  ALLOC(A.pe_i, N); ALLOC(A.pevw_i, N); ALLOC(A.vir_i, N); ALLOC(A.virw_i, N); ALLOC(A.d2w_i, N);
  ALLOC(A.cnt_vv_i, N); ALLOC(A.cnt_vw_i, N);
  ALLOC(A.occ, std::max<size_t>(pores.size(), 1));
  ALLOC(A.ads, (size_t)groups);
  ALLOC(A.prof, (size_t)prof);
  {
    long long chunks = 1;
    for (int r = 0; r < n_reps; ++r)
      chunks = std::max<long long>(chunks, (c->rh[r].n_vap + 1023) / 1024);
    A.rep_chunks = (int32_t)chunks;
  }
  ALLOC(A.rep_part, (size_t)n_reps * A.rep_chunks * 8);
  {
    int mp = 1;
    for (int r = 0; r < n_reps; ++r) mp = std::max(mp, (int)c->rh[r].n_pores);
    A.max_pores = mp;
  }
  ALLOC(A.pore_part, (size_t)n_reps * A.rep_chunks * A.max_pores);
  ALLOC(A.pore_press, std::max<size_t>(pores.size(), 1));
  ALLOC(A.rep_sums, (size_t)n_reps * 8);
  ALLOC(c->bad_row, 1);
#undef ALLOC
  cudaError_t e = cudaMallocHost(&c->status_host, 3 * sizeof(int32_t));
  if (e != cudaSuccess) return bail(fail(c, MD_ENOMEM, "pinned status word"));
  c->status_host[0] = 0;
  c->status_host[1] = kNoBadRow;
  e = cudaEventCreateWithFlags(&c->status_event, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(fail(c, MD_ECUDA, cudaGetErrorString(e)));

  auto up = [&](void* dst, const void* src, size_t bytes) -> md_status {
    if (bytes == 0) return MD_OK;
    CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return MD_OK;
  };
  // vapour in caller order
  std::vector<dvec4> pos(N), vel(N);
  std::vector<int32_t> id(N), rep(N);
  for (int r = 0; r < n_reps; ++r) {
    const md_system* s = &systems[r];
    const int off = c->reps[r].vap_off;
    for (int64_t i = 0; i < s->n_vapor; ++i) {
      pos[off + i] = make_dvec4(s->x0[3 * i], s->x0[3 * i + 1], s->x0[3 * i + 2], 0.0);
      vel[off + i] = make_dvec4(s->v0[3 * i], s->v0[3 * i + 1], s->v0[3 * i + 2], 0.0);
      id[off + i] = (int32_t)i;
      rep[off + i] = r;
    }
  }
  if ((st = up(A.pos, pos.data(), N * sizeof(dvec4))) != MD_OK) return bail(st);
  if ((st = up(A.vel, vel.data(), N * sizeof(dvec4))) != MD_OK) return bail(st);
  if ((st = up(A.id, id.data(), N * sizeof(int32_t))) != MD_OK) return bail(st);
  if ((st = up(A.rep, rep.data(), N * sizeof(int32_t))) != MD_OK) return bail(st);
  if ((st = up(A.wpos, wpos.data(), wpos.size() * sizeof(dvec4))) != MD_OK) return bail(st);
  if ((st = up(A.wlpos, wlpos.data(), wlpos.size() * sizeof(float4))) != MD_OK) return bail(st);
  if ((st = up(A.wlpos_lo, wlpos_lo.data(), wlpos_lo.size() * sizeof(float4))) != MD_OK)
    return bail(st);
  if ((st = up(A.wstart, wstart.data(), wstart.size() * sizeof(int32_t))) != MD_OK) return bail(st);
  if ((st = up(cell_rep_d, cell_rep.data(), cell_rep.size() * sizeof(int32_t))) != MD_OK)
    return bail(st);
  if ((st = up(row_cell_d, row_cell.data(), row_cell.size() * sizeof(int32_t))) != MD_OK)
    return bail(st);
  if ((st = up(wnear_d, wnear.data(), wnear.size() * sizeof(int32_t))) != MD_OK) return bail(st);
  std::vector<float4> wxf;
  if (A.wxf) {
    wxf.resize(nw_tot);
    for (long long k = 0; k < nw_tot; ++k)
      wxf[k] = make_float4((float)wpos[k].x, (float)wpos[k].y, (float)wpos[k].z, 0.f);
    if ((st = up(const_cast<float4*>(A.wxf), wxf.data(), wxf.size() * sizeof(float4))) != MD_OK)
      return bail(st);
  }
  if ((st = up(reps_d, c->reps.data(), c->reps.size() * sizeof(RepDev))) != MD_OK) return bail(st);
  if ((st = up(ctr_d, ctr.data(), ctr.size() * sizeof(double))) != MD_OK) return bail(st);
  if ((st = up(pores_d, pores.data(), pores.size() * sizeof(PoreDev))) != MD_OK) return bail(st);
  // the host staging vectors above die at return: wait for the copies first
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if ((st = rebuild_and_forces(c)) != MD_OK) return bail(st);
  *out = c;
  return MD_OK;
}

}  // namespace

extern "C" {

const char* md_status_string(md_status s) {
  switch (s) {
    case MD_OK: return "ok";
    case MD_EINVAL: return "invalid argument";
    case MD_ENOMEM: return "out of memory";
    case MD_ECUDA: return "CUDA error";
    case MD_EOVERFLOW: return "neighbour list or cell capacity exceeded";
    case MD_EUNSTABLE: return "unstable motion (non-finite or out-of-box position)";
    case MD_ETIMEOUT: return "device wait timed out";
    case MD_EBOUNDS: return "index out of bounds (checked build)";
  }
  return "unknown status";
}

const char* md_last_error(const md_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

md_status md_create(const md_system* sys, const md_potential* pot, void* stream, md_ctx** out) {
  return create_impl(sys, 1, pot, stream, out);
}

md_status md_create_batch(const md_system* systems, int32_t n_replicas, const md_potential* pot,
                          void* stream, md_ctx** out) {
  return create_impl(systems, n_replicas, pot, stream, out);
}

// the flat stream's arrays (force_tpp 64), allocated on first use (their capacity: kFlatPerMol
// entries a molecule, at most a row's); *fresh says whether they are new (then the stream must be
// filled by a rebuild, and graphs captured before hold none of them)
md_status ensure_flat(md_ctx* c, bool* fresh) {
  *fresh = false;
  if (c->a.flat_ent) return MD_OK;
  const long long cap = (long long)c->a.n_total * std::min(c->pot.cap, kFlatPerMol);
  uint32_t* ent = nullptr;
  int32_t *own = nullptr, *part = nullptr, *n = nullptr;
  md_status st;
  if ((st = dalloc(c, &ent, (size_t)cap)) != MD_OK) return st;
  if ((st = dalloc(c, &own, (size_t)cap)) != MD_OK) return st;
  if ((st = dalloc(c, &part, (size_t)c->a.n_total / kFlatBlock + 2)) != MD_OK) return st;
  if ((st = dalloc(c, &n, 1)) != MD_OK) return st;
  c->a.flat_own = own;
  c->a.flat_part = part;
  c->a.n_flat = n;
  c->a.flat_cap = cap;
  c->a.flat_ent = ent;
  *fresh = true;
  destroy_graph(c);
  return MD_OK;
}

md_status md_set_tuning(md_ctx* c, const md_tuning* t) {
  if (!c || !t) return MD_EINVAL;
  Tuning nt = c->tun;
  if (t->force_block) {
    if (t->force_block != 128 && t->force_block != 256)
      return fail(c, MD_EINVAL, "force_block must be 128 or 256");
    nt.force_block = t->force_block;
  }
  if (t->force_blocks_per_sm) {
    if (t->force_blocks_per_sm < 1 || t->force_blocks_per_sm > 32)
      return fail(c, MD_EINVAL, "force_blocks_per_sm must be in [1, 32]");
    if (c->mixed) nt.force_blocks_per_sm_mixed = t->force_blocks_per_sm;
    else nt.force_blocks_per_sm_fp64 = t->force_blocks_per_sm;
  }
  if (t->force_tpp) {
    if (t->force_tpp != 1 && t->force_tpp != 2 && t->force_tpp != 4 && t->force_tpp != 8 &&
        t->force_tpp != 16 && t->force_tpp != kFlatTpp &&
        !(t->force_tpp == 32 && !c->mixed && !c->tun.df64))
      return fail(c, MD_EINVAL, "force_tpp must be 1, 2, 4, 8, 16 or 64 (or 32 at FP64)");
    if (c->mixed) nt.tpp_mixed = t->force_tpp;
    else nt.tpp_fp64 = t->force_tpp;
  }
  if (t->order_by_length < 0 || t->order_by_length > 2)
    return fail(c, MD_EINVAL, "order_by_length must be 0 (keep), 1 (on) or 2 (off)");
  if (t->use_graph < 0 || t->use_graph > 2)
    return fail(c, MD_EINVAL, "use_graph must be 0 (keep), 1 (graph) or 2 (plain launches)");
  if (t->steps_per_graph < 0) return fail(c, MD_EINVAL, "steps_per_graph < 0");
  if (t->force_accumulate < 0 || t->force_accumulate > 2)
    return fail(c, MD_EINVAL, "force_accumulate must be 0 (keep), 1 (deterministic) or 2 (atomic)");
  if (t->chunk_walk < 0 || t->chunk_walk > 2)
    return fail(c, MD_EINVAL, "chunk_walk must be 0 (keep), 1 (dynamic) or 2 (static)");
  if (t->chunk_walk) nt.static_chunks = t->chunk_walk == 2 ? 1 : 0;
  if (t->list_build < 0 || t->list_build > 3)
    return fail(c, MD_EINVAL, "list_build must be 0 (keep), 1 (device's choice), 2 (warp per cell) "
                              "or 3 (thread per molecule)");
  if (t->list_build) nt.list_mode = t->list_build - 1;
  if (t->pair_method < 0 || t->pair_method > 4)
    return fail(c, MD_EINVAL, "pair_method must be 0 (keep), 1 (Verlet lists), 2 (all pairs), "
                              "3 (cells) or 4 (small systems)");
  if ((c->mixed || c->tun.df64) && (t->pair_method == 2 || t->pair_method == 4))
    return fail(c, MD_EINVAL, "the all-pairs and small-system methods are FP64-path options");
  if (t->pair_method == 4 && !c->a.xf)
    return fail(c, MD_EINVAL, "the small-system method takes at most " +
                                  std::to_string(kSmallMax) + " molecules");
  if (t->pair_method) {
    nt.all_pairs = t->pair_method == 2 ? 1 : 0;
    nt.cells = t->pair_method == 3 ? 1 : 0;
    nt.small = t->pair_method == 4 ? 1 : 0;
  }
  const bool chosen = c->method_chosen || t->pair_method != 0;
  if (nt.cells && t->force_accumulate == 1)
    return fail(c, MD_EINVAL, "the cell method adds reaction forces by atomics (force_accumulate 2)");
  const int at = nt.cells ? 1
                 : t->force_accumulate ? (t->force_accumulate == 2 ? 1 : 0) : c->tun.atomic_acc;
  if (!at && (c->mixed ? nt.tpp_mixed : nt.tpp_fp64) == kFlatTpp)
    return fail(c, MD_EINVAL, "force_tpp 64 (the flat stream) adds reaction forces by atomics "
                              "(force_accumulate 2)");
  bool relist = t->order_by_length && (t->order_by_length == 1) != (c->tun.lpt != 0);
  if (t->order_by_length) nt.lpt = t->order_by_length == 1;
  relist = relist || at != c->tun.atomic_acc;  // the deterministic form needs the pair map
  relist = relist || nt.all_pairs != c->tun.all_pairs;  // lists fresh when they come back
  relist = relist || nt.cells != c->tun.cells || nt.small != c->tun.small;
  // the packed kernel screens with the FP32 cell-local offsets: refresh them on the way in
  relist = relist || (!c->mixed && (nt.tpp_fp64 >= 32) != (c->tun.tpp_fp64 >= 32));
  // the flat stream's rebuilds keep no processing order, the other kernels' no stream
  relist = relist || ((c->mixed ? nt.tpp_mixed : nt.tpp_fp64) == kFlatTpp) !=
                         ((c->mixed ? c->tun.tpp_mixed : c->tun.tpp_fp64) == kFlatTpp);
  if ((c->mixed ? nt.tpp_mixed : nt.tpp_fp64) == kFlatTpp) {  // the stream is filled at rebuilds
    bool fresh = false;
    md_status st = ensure_flat(c, &fresh);
    if (st != MD_OK) return st;
    relist = relist || fresh;
  }
  nt.atomic_acc = at;
  c->tun = nt;
  c->method_chosen = chosen;
  if (t->use_graph) c->use_graph = t->use_graph == 1 ? 1 : 0;
  if (t->steps_per_graph) c->steps_per_graph = t->steps_per_graph;
  destroy_graph(c);
  // the processing order is built with the lists: rebuild them now
  if (relist) return rebuild_and_forces(c);
  return MD_OK;
}

md_status md_get_tuning(const md_ctx* c, md_tuning* t) {
  if (!c || !t) return MD_EINVAL;
  t->force_block = c->tun.force_block;
  t->force_blocks_per_sm =
      c->mixed ? c->tun.force_blocks_per_sm_mixed : c->tun.force_blocks_per_sm_fp64;
  t->force_tpp = c->mixed ? c->tun.tpp_mixed : c->tun.tpp_fp64;
  t->order_by_length = c->tun.lpt ? 1 : 2;
  t->use_graph = c->use_graph ? 1 : 2;
  t->steps_per_graph = c->steps_per_graph;
  t->force_accumulate = c->tun.atomic_acc ? 2 : 1;
  t->pair_method = c->tun.small ? 4 : c->tun.cells ? 3 : (c->tun.all_pairs ? 2 : 1);
  t->chunk_walk = c->tun.static_chunks ? 2 : 1;
  t->list_build = c->tun.list_mode + 1;
  return MD_OK;
}

md_status md_autotune(md_ctx* c, int32_t trials, md_tuning* best, double* best_us) {
  if (!c) return MD_EINVAL;
  md_status s = sync_status(c);
  if (s != MD_OK) return s;
  trials = std::max(3, std::min(101, trials));
  std::vector<cudaEvent_t> ev(2 * (size_t)trials);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto& f : ev) if (f) cudaEventDestroy(f);
      return fail(c, MD_ECUDA, "cudaEventCreate");
    }
  const Tuning saved = c->tun;
  Tuning bestT = saved;
  double bestv = 1e300;
  md_status st = MD_OK;
  const bool fixed_shape = saved.small;  // the small-system kernel has no shapes to choose
  if (saved.atomic_acc && !saved.all_pairs && !saved.cells && !fixed_shape) {
    bool fresh = false;  // the flat stream is a candidate: its arrays, filled by the rebuilds below
    if ((s = ensure_flat(c, &fresh)) != MD_OK) {
      for (auto& e : ev) cudaEventDestroy(e);
      return s;
    }
  }
  const int tpps[7] = {1, 2, 4, 8, 16, 32, kFlatTpp}, bpss[4] = {1, 2, 4, 8},
            blocks[2] = {128, 256};
  auto time_shape = [&](const Tuning& t) -> bool {
    launch_forces(c->a, c->pot, c->mixed, false, false, t, c->stream);  // warm-up
    for (int k = 0; k < trials; ++k) {
      cudaEventRecord(ev[2 * k], c->stream);
      launch_forces(c->a, c->pot, c->mixed, false, false, t, c->stream);
      cudaEventRecord(ev[2 * k + 1], c->stream);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      return false;
    std::vector<float> ms(trials);
    for (int k = 0; k < trials; ++k) cudaEventElapsedTime(&ms[k], ev[2 * k], ev[2 * k + 1]);
    std::nth_element(ms.begin(), ms.begin() + trials / 2, ms.end());
    const double us = 1e3 * ms[trials / 2];
    if (us < bestv) {
      bestv = us;
      bestT = t;
    }
    return true;
  };
  // the method is the caller's once chosen: a context on the cell method times its shapes alone,
  // one on the Verlet lists times theirs; otherwise both are timed (the cell method in the atomic
  // form only)
  if (fixed_shape && !time_shape(saved)) st = fail(c, MD_ECUDA, "autotune launch failed");
  for (int lpt = 1; lpt >= 0 && st == MD_OK && !saved.cells && !fixed_shape; --lpt) {
    c->tun = saved;
    c->tun.lpt = lpt;
    c->tun.cells = 0;
    c->tun.flat_fill = c->a.flat_ent ? 1 : 0;  // every list kernel's inputs, for the timings
    if ((st = rebuild_and_forces(c)) != MD_OK) break;
    for (int tp : tpps) {
      // the packed kernels are the FP64 path's
      if (tp == 32 && (c->mixed || c->tun.df64)) continue;
      // the flat stream is an atomic form
      if (tp == kFlatTpp && (!c->tun.atomic_acc || c->tun.all_pairs)) continue;
      for (int bp : bpss)
        for (int bk : blocks) {
          // the all-pairs kernel has a fixed shape: time it once
          if (c->tun.all_pairs && (tp != tpps[0] || bp != bpss[0] || bk != blocks[0] || !lpt))
            continue;
          for (int walk = 0; walk < 2 && st == MD_OK; ++walk) {
            // the static walk is a shape of the atomic list kernels of force_tpp 1 to 16
            if (walk && !(c->tun.atomic_acc && tp < 32 && !c->tun.all_pairs)) continue;
            // the flat stream splits the whole list: one processing order is enough
            if (tp == kFlatTpp && !lpt) continue;
            Tuning t = c->tun;
            t.force_block = bk;
            t.static_chunks = walk;
            if (c->mixed) {
              t.tpp_mixed = tp;
              t.force_blocks_per_sm_mixed = bp;
            } else {
              t.tpp_fp64 = tp;
              t.force_blocks_per_sm_fp64 = bp;
            }
            if (!time_shape(t)) st = fail(c, MD_ECUDA, "autotune launch failed");
          }
        }
    }
  }
  // the cell method (no lists) is a further form of the atomic half-pair evaluation
  if (st == MD_OK && !saved.all_pairs && !fixed_shape &&
      (saved.cells || (saved.atomic_acc && !c->method_chosen))) {
    c->tun = saved;
    c->tun.cells = 1;
    c->tun.atomic_acc = 1;
    if ((st = rebuild_and_forces(c)) == MD_OK)
      for (int bp : {1, 2, 4})
        for (int bk : blocks) {
          Tuning t = c->tun;
          t.force_block = bk;
          if (c->mixed) t.force_blocks_per_sm_mixed = bp;
          else t.force_blocks_per_sm_fp64 = bp;
          if (!time_shape(t)) {
            st = fail(c, MD_ECUDA, "autotune launch failed");
            break;
          }
        }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != MD_OK) {
    c->tun = saved;
    return st;
  }
  c->tun = bestT;
  c->tun.flat_fill = 0;
  destroy_graph(c);
  // lists (and their processing order) for the chosen shape; forces at the same positions
  if ((st = rebuild_and_forces(c)) != MD_OK) return st;
  if (best) md_get_tuning(c, best);
  if (best_us) *best_us = bestv;
  return MD_OK;
}

md_status md_check_barrier_timeout(md_ctx* c, double* seconds) {
  if (!c) return MD_EINVAL;
  md_status s = sync_status(c);
  if (s != MD_OK) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, MD_ECUDA, "cudaEventCreate");
  }
  cudaEventRecord(e0, c->stream);
  launch_barrier_check(c->a, c->pot, c->stream);
  cudaEventRecord(e1, c->stream);
  const cudaError_t le = cudaGetLastError();
  s = le == cudaSuccess ? sync_status(c) : MD_ECUDA;
  float ms = 0.f;
  if (le == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess) return fail(c, MD_ECUDA, cudaGetErrorString(le));
  // the status word and the barrier's count back as they were: the context goes on
  CUDA_TRY(c, cudaMemsetAsync(c->a.status, 0, 2 * sizeof(int32_t), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->a.bar_arrive, 0, sizeof(unsigned long long), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->last_status_bits = 0;
  c->err.clear();
  if (seconds) *seconds = ms * 1e-3;
  if (s != MD_ETIMEOUT)
    return fail(c, MD_ECUDA, std::string("the bounded wait did not report its timeout (status: ") +
                                 md_status_string(s) + ")");
  return MD_OK;
}

md_status md_step(md_ctx* c, int64_t n) {
  if (!c) return MD_EINVAL;
  if (n < 0) return fail(c, MD_EINVAL, "negative step count");
  // pick up the status copied at the end of the previous call, if it has landed
  if (c->status_pending && cudaEventQuery(c->status_event) == cudaSuccess) {
    c->status_pending = false;
    c->last_status_bits = *c->status_host;
  }
  md_status prev = device_status(c);
  if (prev != MD_OK) return prev;
  int64_t left = n;
  if (c->tun.small) {  // whole steps in cooperative launches of at most 1000 steps each
    for (; left > 0; left -= std::min<int64_t>(left, 1000))
      launch_small_steps(c->a, c->pot, c->tun, (int)std::min<int64_t>(left, 1000), c->stream);
  }
  if (c->use_graph && n >= c->steps_per_graph && left > 0) {
    if (c->graph_steps != c->steps_per_graph) {
      md_status s = build_graph(c, c->steps_per_graph);
      if (s != MD_OK) return s;
    }
    while (left >= c->graph_steps) {
      CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, c->stream));
      left -= c->graph_steps;
    }
  }
  for (int64_t k = 0; k < left; ++k) enqueue_step(c);
  CUDA_TRY(c, cudaGetLastError());
  c->steps_done += n;
  if (!c->status_pending) {
    CUDA_TRY(c, cudaMemcpyAsync(c->status_host, c->a.status, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, c->stream));
    c->bytes_d2h += sizeof(int32_t);
    CUDA_TRY(c, cudaEventRecord(c->status_event, c->stream));
    c->status_pending = true;
  }
  return MD_OK;
}

md_status md_sync(md_ctx* c) {
  if (!c) return MD_EINVAL;
  return sync_status(c);
}

// molecules of replica r (or of every replica, r = -1): first record and count
static void replica_range(const md_ctx* c, int32_t r, int* off, int* n) {
  if (r < 0) {
    *off = 0;
    *n = c->a.n_total;
  } else {
    *off = c->reps[r].vap_off;
    *n = c->reps[r].n_vap;
  }
}

static bool check_replica_or_all(md_ctx* c, int32_t r) { return c && r >= -1 && r < c->n_reps; }

// records -> caller-order rows on the device -> one copy into the caller's array
static md_status fetch_rows(md_ctx* c, int32_t r, const dvec4* dsrc, double* stage, double* out) {
  int off, n;
  replica_range(c, r, &off, &n);
  launch_store_rows(c->a, dsrc, stage, off, n, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  if (n)
    CUDA_TRY(c, cudaMemcpyAsync(out, stage + 3 * (size_t)off, 3 * (size_t)n * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  c->bytes_d2h += (int64_t)(3 * (size_t)n * sizeof(double));
  return MD_OK;
}

md_status md_get_state(md_ctx* c, int32_t r, double* x, double* v) {
  if (!check_replica_or_all(c, r)) return fail(c, MD_EINVAL, "bad replica");
  md_status s = sync_status(c);
  if (s != MD_OK && s != MD_EOVERFLOW && s != MD_EUNSTABLE && s != MD_ETIMEOUT) return s;
  md_status t;
  if (v) launch_settle(c->a, c->pot, c->stream);
  if (x && (t = fetch_rows(c, r, c->a.pos, c->stage_x, x)) != MD_OK) return t;
  if (v && (t = fetch_rows(c, r, c->a.vel, c->stage_v, v)) != MD_OK) return t;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return s;
}

md_status md_get_forces(md_ctx* c, int32_t r, double* f) {
  if (!check_replica_or_all(c, r) || !f) return fail(c, MD_EINVAL, "bad replica or NULL output");
  // the status word and the rows behind one synchronisation
  md_status t = enqueue_status(c);
  if (t != MD_OK) return t;
  if ((t = fetch_rows(c, r, c->a.frc, c->stage_x, f)) != MD_OK) return t;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return status_after_sync(c);
}

md_status md_set_state(md_ctx* c, int32_t r, const double* x, const double* v) {
  if (!check_replica_or_all(c, r) || !x || !v)
    return fail(c, MD_EINVAL, "bad replica or NULL input");
  md_status s = sync_status(c);
  if (s != MD_OK) return s;
  int off, n;
  replica_range(c, r, &off, &n);
  // what the last step owes (its second half-kick, its thermostat) is paid before the load resets
  // the flags (a state-preserving step, taken whether or not the rows pass their check)
  launch_settle(c->a, c->pot, c->stream);
  // the list methods keep the stored order and rebuild only where the skin test asks for it; the
  // all-pairs and small-system methods keep no lists
  const bool keep = !c->tun.all_pairs && !c->tun.small;
  if (n) {
    const size_t bytes = 3 * (size_t)n * sizeof(double);
    CUDA_TRY(c, cudaMemcpyAsync(c->stage_x + 3 * (size_t)off, x, bytes, cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->stage_v + 3 * (size_t)off, v, bytes, cudaMemcpyHostToDevice,
                                c->stream));
    c->bytes_h2d += (int64_t)(2 * bytes);
    // every row is checked on the device (inside its replica's box; planar replicas in the
    // plane) before the load, which leaves the state untouched if any row fails
    CUDA_TRY(c, cudaMemsetAsync(c->bad_row, 0x7f, sizeof(int32_t), c->stream));
    if (keep) {  // the load raises the rebuild flags as a step's skin check does
      CUDA_TRY(c, cudaMemsetAsync(c->a.force_rebuild, 0, sizeof(int), c->stream));
      CUDA_TRY(c, cudaMemsetAsync(c->a.rep_disp2, 0,
                                  sizeof(unsigned long long) * (size_t)c->n_reps, c->stream));
    }
    launch_load_state(c->a, c->pot, c->stage_x, c->stage_v, off, n, c->bad_row, keep, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(c->status_host + 1, c->bad_row, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, c->stream));
    c->bytes_d2h += sizeof(int32_t);
  }
  md_status st;
  if (keep) {
    // the check's row and the load's rebuild flag read back together; the rebuild chain is
    // launched only when some replica asks for it, and forces only after a load that happened
    c->status_host[2] = 0;
    if (n) {
      CUDA_TRY(c, cudaMemcpyAsync(c->status_host + 2, c->a.force_rebuild, sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, c->stream));
      c->bytes_d2h += sizeof(int32_t);
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    if (n && c->status_host[1] != kNoBadRow) {
      st = sync_status(c);  // nothing was loaded: the forces stand
    } else {
      if (c->status_host[2]) launch_rebuild(c->a, c->pot, c->tun, c->mixed, c->stream);
      launch_forces(c->a, c->pot, c->mixed, false, false, c->tun, c->stream);
      CUDA_TRY(c, cudaGetLastError());
      st = sync_status(c);
    }
  } else {
    st = rebuild_and_forces(c);  // (waits for the stream, the check's row included)
  }
  const int32_t bad = c->status_host[1];
  c->status_host[1] = kNoBadRow;
  if (n && bad != kNoBadRow) {
    const int row = off + bad / 3;
    int rr = 0;
    while (rr + 1 < c->n_reps && c->reps[rr + 1].vap_off <= row) ++rr;
    static const char* const why[3] = {" outside the box", " leaves the plane y = 0",
                                       " has a non-finite velocity"};
    return fail(c, MD_EINVAL, "replica " + std::to_string(rr) + ": molecule " +
                                  std::to_string(row - c->reps[rr].vap_off) + why[bad % 3]);
  }
  return st;
}

md_status md_observables(md_ctx* c, int32_t r, md_obs* out, int64_t* occupancy, int64_t* adsorbed,
                         int64_t* profile, double* pore_pressure) {
  if (!check_replica(c, r) || !out) return fail(c, MD_EINVAL, "bad replica or NULL output");
  md_status s = sync_status(c);
  if (s != MD_OK) return s;
  Arrays& A = c->a;
  CUDA_TRY(c, cudaMemsetAsync(A.occ, 0, std::max<size_t>(c->pores_total, 1) * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(A.ads, 0, c->groups_total * 8, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(A.prof, 0, std::max<size_t>(c->prof_total, 1) * 8, c->stream));
  launch_settle(A, c->pot, c->stream);  // kinetic energy at v(t+dt), after the thermostat
  launch_forces(A, c->pot, c->mixed, true, false, c->tun, c->stream);
  launch_observables(A, c->pot, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  const RepDev& R = c->reps[r];
  const ReplicaHost& H = c->rh[r];
  double sums[8];
  unsigned long long nreb = 0, pc = 0;
  long long step = 0;
  int32_t mv = 0;
  std::vector<unsigned long long> occ(std::max(H.n_pores, 1)), ads(H.n_groups),
      prof((size_t)H.n_groups * H.n_bins);
  CUDA_TRY(c, cudaMemcpyAsync(sums, A.rep_sums + 8 * r, 8 * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&nreb, A.n_rebuilds, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&pc, A.pair_count, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&step, A.step, 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&mv, A.max_nb, 4, cudaMemcpyDeviceToHost, c->stream));
  if (H.n_pores)
    CUDA_TRY(c, cudaMemcpyAsync(occ.data(), A.occ + R.pore_off, H.n_pores * 8,
                                cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(ads.data(), A.ads + R.group_off, H.n_groups * 8,
                              cudaMemcpyDeviceToHost, c->stream));
  if (!prof.empty())
    CUDA_TRY(c, cudaMemcpyAsync(prof.data(), A.prof + R.prof_off, prof.size() * 8,
                                cudaMemcpyDeviceToHost, c->stream));
  if (pore_pressure && H.n_pores)
    CUDA_TRY(c, cudaMemcpyAsync(pore_pressure, A.pore_press + R.pore_off, H.n_pores * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::memset(out, 0, sizeof(*out));
  out->step = step;
  out->n_vapor = H.n_vap;
  out->n_wall = H.n_wall;
  out->ke = sums[0];
  out->pe_vv = sums[1];
  out->pe_vw = sums[2];
  out->pe = sums[1] + sums[2];
  out->T = H.n_vap ? 2.0 * sums[0] / ((double)c->reps[r].dims * (double)H.n_vap) : 0.0;
  out->virial_vv = sums[3];
  out->virial_vw = sums[4];
  out->pairs_vv = (int64_t)std::llround(sums[5]) / 2;
  out->pairs_vw = (int64_t)std::llround(sums[6]);
  out->n_groups = H.n_groups;
  out->n_bins = H.n_bins;
  out->n_rebuilds = (int64_t)nreb;
  out->pair_evals_total = (int64_t)(pc / 2);
  out->max_list_used = mv;
  out->list_capacity = c->pot.cap;
  for (int q = 0; q < H.n_pores; ++q) {
    out->occupancy += (int64_t)occ[q];
    if (occupancy) occupancy[q] = (int64_t)occ[q];
  }
  for (int g = 0; g < H.n_groups; ++g) {
    out->adsorbed += (int64_t)ads[g];
    if (adsorbed) adsorbed[g] = (int64_t)ads[g];
  }
  if (profile)
    for (size_t k = 0; k < prof.size(); ++k) profile[k] = (int64_t)prof[k];
  return sync_status(c);
}

md_status md_compute_forces(md_ctx* c) {
  if (!c) return MD_EINVAL;
  md_status prev = device_status(c);
  if (prev != MD_OK) return prev;
  launch_forces(c->a, c->pot, c->mixed, false, false, c->tun, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  return MD_OK;
}

md_status md_pair_pass(md_ctx* c) {
  if (!c) return MD_EINVAL;
  md_status prev = device_status(c);
  if (prev != MD_OK) return prev;
  launch_pair_pass(c->a, c->pot, c->mixed, c->tun, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  return MD_OK;
}

md_status md_rebuild_lists(md_ctx* c) {
  if (!c) return MD_EINVAL;
  if (c->tun.all_pairs || c->tun.small)
    return fail(c, MD_EINVAL, "the all-pairs and small-system methods keep no lists");
  md_status prev = device_status(c);
  if (prev != MD_OK) return prev;
  // every replica rebuilds (all-ones bytes: the largest displacement pattern)
  CUDA_TRY(c, cudaMemsetAsync(c->a.force_rebuild, 0x01, sizeof(int), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->a.rep_disp2, 0xff, sizeof(unsigned long long) * (size_t)c->n_reps,
                              c->stream));
  launch_rebuild(c->a, c->pot, c->tun, c->mixed, c->stream);
  // the current positions are now every molecule's reference: nothing is due (the flags a pair
  // kernel clears after a chain)
  CUDA_TRY(c, cudaMemsetAsync(c->a.force_rebuild, 0, sizeof(int), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->a.rep_disp2, 0, sizeof(unsigned long long) * (size_t)c->n_reps,
                              c->stream));
  CUDA_TRY(c, cudaGetLastError());
  return MD_OK;
}

md_status md_transfer_bytes(const md_ctx* c, int64_t* h2d, int64_t* d2h) {
  if (!c) return MD_EINVAL;
  if (h2d) *h2d = c->bytes_h2d;
  if (d2h) *d2h = c->bytes_d2h;
  return MD_OK;
}

md_status md_get_wall(md_ctx* c, int32_t r, double* w) {
  if (!check_replica(c, r) || !w) return fail(c, MD_EINVAL, "bad replica or NULL output");
  const std::vector<double>& W = c->rh[r].wall;
  if (!W.empty()) std::memcpy(w, W.data(), W.size() * sizeof(double));
  return MD_OK;
}

md_status md_get_sizes(const md_ctx* c, int32_t r, int64_t* n_vapor, int64_t* n_wall,
                       int32_t* n_groups, int32_t* n_bins) {
  if (!c || r < 0 || r >= c->n_reps) return MD_EINVAL;
  const ReplicaHost& H = c->rh[r];
  if (n_vapor) *n_vapor = H.n_vap;
  if (n_wall) *n_wall = H.n_wall;
  if (n_groups) *n_groups = H.n_groups;
  if (n_bins) *n_bins = H.n_bins;
  return MD_OK;
}

int64_t md_kernel_launches(const md_ctx* c) {
  if (!c || !c->a.launch_count) return 0;
  unsigned long long n = 0;
  if (cudaMemcpyAsync(&n, c->a.launch_count, sizeof(n), cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (int64_t)n;
}

void md_destroy(md_ctx* c) {
  if (!c) return;
  if (c->stream || !c->allocs.empty()) cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  for (void* p : c->allocs) cudaFree(p);
  if (c->status_host) cudaFreeHost(c->status_host);
  if (c->status_event) cudaEventDestroy(c->status_event);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  if (c->aux) cudaStreamDestroy(c->aux);
  delete c;
}

}  // extern "C"
