// md_kernels.cu -- CUDA kernels (sm_103a) of the pore / water-vapour MD step.
//
// One MD step (Sec. 2 velocity Verlet, Figs. 1-4 of arXiv:1812.07993), all replicas per launch:
//   k_integrate_first   the previous step's owed second half-kick (Fig. 3) and Berendsen scaling
//                       (Fig. 4), then half-kick + drift (Fig. 2), z reflection, hard-wall
//                       reflection, x/y wrap, skin check; its last block decides whether lists are
//                       rebuilt (a CUDA-graph conditional node) and whether this step owes a
//                       thermostat
//   rebuild chain       only when a molecule moved >= skin/2 since its replica's last build, and
//                       only for the replicas near their limit:
//                         k_cell_clear -> k_cell_count -> k_scan_* -> k_scatter -> k_permute ->
//                         k_list_build (warp per cell; list-length counts, whose scan its last
//                         block does) -> k_order_assign [-> k_fwd_build]
//   pair forces         Lennard-Jones forces at r(t+dt) (Eq. 2, Fig. 1) and the second half-kick
//                       (Fig. 3), in one of:
//                         FP64 half list + slot-and-gather, the kick fused into the gather;
//                         FP64 half list with atomic reaction forces (lanes per molecule, or
//                         the compacted form: FP32 screen, per-warp queue of FP64 pair terms);
//                         mixed precision, full list, the kick fused in;
//                         mixed precision, half list with atomic reaction forces;
//                         FP64 context, double-float pair terms: full list (the kick fused
//                         in) or half list with atomic reaction forces.
//                       The atomic forms defer the kick into the next first half-kick
//                       (k_kick_pending settles it before the thermostat or any velocity read).
//   Berendsen scaling (Fig. 4) of a thermostat step is paid by the next step's k_integrate_first
//                       (a grid barrier on those steps only), or, before a state read, by
//                       k_kick_pending / k_thermo_partial / k_thermo_lambda / k_thermo_scale
// One kernel waits on other blocks: k_integrate_first, at a bounded grid barrier, on steps that
// owe a thermostat; its grid holds only as many blocks as the SMs keep resident at once. Elsewhere
// one block finishes a launch's work (the last-block pattern): the one whose report comes in last.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void count_launch(const Arrays& a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.launch_count, 1ull);
}

__device__ __forceinline__ bool halted(const Arrays& a) {
  return *reinterpret_cast<volatile const int32_t*>(a.status) != 0;
}

// lists are rebuilt when the host asks for it or when some molecule has moved at least skin/2
// since the last build (k_integrate_first raises the same flag); the pair kernel clears it
__device__ __forceinline__ bool need_rebuild(const Arrays& a, const PotDev& p) {
  return *reinterpret_cast<volatile const int32_t*>(a.force_rebuild) != 0;
}

// replica r rebuilds its lists in this chain: some molecule of it moved past the grouping
// threshold (0.6 skin/2) since its last build -- the chain runs only once some molecule somewhere
// reached skin/2 -- or the host asked. The other replicas keep their order, cells and lists;
// grouping near-due replicas into the same chain keeps chains rare when replicas are many.
__device__ __forceinline__ bool rep_rebuilds(const Arrays& a, int r) {
  return a.rep_disp2[r] != 0ull;
}

// the pair kernels clear the rebuild flags once the chain has run
__device__ __forceinline__ void clear_rebuild_flags(const Arrays& a) {
  if (blockIdx.x != 0) return;
  if (threadIdx.x == 0) *a.force_rebuild = 0;
  for (int r = threadIdx.x; r < a.n_reps; r += blockDim.x) a.rep_disp2[r] = 0ull;
}

// periodic image of a coordinate difference of two wrapped positions (|d| < L): the high word of
// |d| is compared against the high word of L/2 -- an integer test, no FP64 instruction. Pairs in a
// list are either closer than the list radius or further than L minus it, far from L/2.
__device__ __forceinline__ double image_hi(double d, double L, uint32_t thr) {
  const int hw = __double2hiint(d);
  const double sh = (uint32_t)(hw & 0x7fffffff) >= thr ? (hw < 0 ? L : -L) : 0.0;
  return d + sh;  // one FP64 add; the shift is chosen by integer selects
}

// exact periodic wrap of a difference (compare form)
__device__ __forceinline__ double wrap_diff(double d, double L, double h) {
  if (d >= h) return d - L;
  if (d < -h) return d + L;
  return d;
}

__device__ __forceinline__ int pack_home(int ix, int iy, int iz) {
  return ix | (iy << 10) | (iz << 20);
}

// position relative to the centre of the home cell (centres from the per-replica table), the
// periodic wrap decided by integer tests, in FP64
__device__ __forceinline__ void local_offset_d(const Arrays& a, const RepDev& R, const dvec4& x,
                                               int home, double& lx, double& ly, double& lz) {
  const int ix = home & 1023, iy = (home >> 10) & 1023, iz = (home >> 20) & 1023;
  const double* __restrict__ ctr = a.cell_ctr + R.ctr_off;
  lx = x.x - ctr[ix];
  ly = x.y - ctr[R.ncx + iy];
  lz = x.z - ctr[R.ncx + R.ncy + iz];
  // d >= L/2 and d < -L/2 as bit-pattern tests (-d flips the sign bit); L/2 > 0
  const long long sgn = (long long)0x8000000000000000ull;
  const long long hxb = __double_as_longlong(R.hx), hyb = __double_as_longlong(R.hy);
  if (__double_as_longlong(lx) >= hxb) lx -= R.Lx;
  else if ((__double_as_longlong(lx) ^ sgn) > hxb) lx += R.Lx;
  if (__double_as_longlong(ly) >= hyb) ly -= R.Ly;
  else if ((__double_as_longlong(ly) ^ sgn) > hyb) ly += R.Ly;
}

// the offset rounded to FP32, for the list test, the screens, the mixed terms and the skin check
__device__ __forceinline__ float4 local_offset(const Arrays& a, const RepDev& R, const dvec4& x,
                                               int home) {
  double lx, ly, lz;
  local_offset_d(a, R, x, home, lx, ly, lz);
  return make_float4(narrow_f64(lx), narrow_f64(ly), narrow_f64(lz), 0.f);
}

// 1/x for a positive normal double x in [2^-126, 2^127] (squared distances), without an FP64
// conversion: x's exponent and leading 20 mantissa bits are rebuilt as an FP32 number with integer
// operations, its correctly rounded FP32 reciprocal (relative error < 2^-19.9) is widened back to
// FP64 the same way, and one third-order Newton step y + y (e + e^2), e = 1 - x y, cubes the error
// (within an ulp of 1/x). Three FP64 FMAs in all.
__device__ __forceinline__ double rcp_nr(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const float xf = __uint_as_float((hi << 3) - (896u << 23));  // exponent bias 1023 -> 127
  const unsigned yb = __float_as_uint(__frcp_rn(xf));
  const double y = __hiloint2double((int)((yb >> 3) + (896u << 20)), (int)(yb << 29));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// -x by flipping the sign bit (an integer operation)
__device__ __forceinline__ double neg_bits(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// comparisons against a positive threshold t by bit patterns (integer instructions): finite IEEE
// doubles order like their patterns read as signed 64-bit integers when t > 0
__device__ __forceinline__ bool gt_pos(double x, double t) {
  return __double_as_longlong(x) > __double_as_longlong(t);
}
__device__ __forceinline__ bool ge_pos(double x, double t) {
  return __double_as_longlong(x) >= __double_as_longlong(t);
}
// |x| <= t; false for NaN
__device__ __forceinline__ bool abs_le(double x, double t) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffll) <= __double_as_longlong(t);
}

// (code - 1) * lc for a 2-bit cell-offset code (0, 1, 2: one cell down, the same cell, one cell up),
// by selects: an int-to-float conversion would run on the FP64 pipe's rate
__device__ __forceinline__ float cell_shift(uint32_t code, float lc) {
  return code == 0u ? -lc : (code == 2u ? lc : 0.f);
}

// the offset as a double-float pair: hi = FP32 rounding (lpos), lo = FP32 rounding of the rest
__device__ __forceinline__ void local_offset_df(const Arrays& a, const RepDev& R, const dvec4& x,
                                                int home, float4& hi, float4& lo) {
  double lx, ly, lz;
  local_offset_d(a, R, x, home, lx, ly, lz);
  hi = make_float4(narrow_f64(lx), narrow_f64(ly), narrow_f64(lz), 0.f);
  lo = make_float4(narrow_f64(lx - widen_f32(hi.x)), narrow_f64(ly - widen_f32(hi.y)),
                   narrow_f64(lz - widen_f32(hi.z)), 0.f);
}

// ---- double-float ("double-word") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, two
// FP32 numbers carrying ~48 significant bits. The building blocks are the error-free
// transformations of Dekker (1971) and Knuth (TAOCP vol. 2) -- Fast2Sum, TwoSum, TwoProd through
// an FMA -- combined as in Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic" (ACM TOMS 44, 2017); every operation runs on the FP32
// pipe, which issues 64 times the FP64 rate on this part.
struct dword {
  float hi, lo;
};
// Fast2Sum (Dekker): a + b = s + e exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ dword fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
// TwoSum (Knuth): a + b = s + e exactly, any order of magnitude
__device__ __forceinline__ dword two_sum(float a, float b) {
  const float s = a + b;
  const float bp = s - a;
  return {s, (a - (s - bp)) + (b - bp)};
}
// TwoProd: a * b = p + e exactly, the error from one FMA
__device__ __forceinline__ dword two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
// double-word + double-word (the "sloppy" sum: error below 2^-46 (|a| + |b|))
__device__ __forceinline__ dword dw_add(dword a, dword b) {
  const dword s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
// double-word * double-word (error below 2^-45 |a b|)
__device__ __forceinline__ dword dw_mul(dword a, dword b) {
  dword p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dword dw_sqr(dword a) {
  dword p = two_prod(a.hi, a.hi);
  p.lo = fmaf(a.hi + a.hi, a.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// 1/a for a > 0: the correctly rounded FP32 reciprocal y of a.hi, then one Newton step
// y + y (1 - a y) with the residual 1 - a y formed from an exact product (error ~2^-46)
__device__ __forceinline__ dword dw_rcp(dword a) {
  const float y = __frcp_rn(a.hi);
  const dword p = two_prod(a.hi, y);           // a.hi y = p.hi + p.lo exactly; p.hi ~ 1
  const float r = ((1.0f - p.hi) - p.lo) - a.lo * y;
  return fast_two_sum(y, y * r);
}
// the double-word value to FP64: both parts widened exactly, one FP64 add
__device__ __forceinline__ double dw_to_double(dword a) {
  return widen_f32(a.hi) + widen_f32(a.lo);
}

// error-free transformation s + x = t + e (Knuth's TwoSum); the error is collected in c
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float e = (s - (t - bp)) + (x - bp);
  s = t;
  c += e;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

inline int nblocks(long long n, int b) { return n > 0 ? (int)((n + b - 1) / b) : 1; }

// ------------------------------------------------------------------------------------------------
// Hard walls (the paper's reflecting pore walls, Sec. 4 and Sec. 5): the slab |z| < h minus the
// pores is solid. A molecule that ended the drift inside it (r, from r0) is mirrored in the face it
// crossed: the slab face on its side when it came from outside the slab, else the side walls and
// the floor of the pore it came from (prism |dx| = r0, |dy| = r1, z = floor; slit |dy| = w/2).
__device__ bool in_any_pore(const Arrays& a, const RepDev& R, double x, double y, double z) {
  for (int q = 0; q < R.n_pores; ++q) {
    const PoreDev& P = a.pores[R.pore_off + q];
    if (in_pore(P.kind, P.r0, P.r1, P.r_cavity, P.width, wrap_diff(x - P.cx, R.Lx, R.hx),
                wrap_diff(y - P.cy, R.Ly, R.hy), z, R.slab_half))
      return true;
  }
  return false;
}

__device__ __noinline__ void reflect_solid(const Arrays& a, const RepDev& R, const dvec4& r0, dvec4& r,
                              dvec4& v) {
  const double h = R.slab_half;
  if (!(fabs(r.z) < h) || in_any_pore(a, R, r.x, r.y, r.z)) return;
  if (fabs(r0.z) >= h) {
    const double face = r0.z > 0.0 ? h : -h;
    r.z = 2.0 * face - r.z;
    v.z = -v.z;
    return;
  }
  for (int q = 0; q < R.n_pores; ++q) {
    const PoreDev& P = a.pores[R.pore_off + q];
    const double dx0 = wrap_diff(r0.x - P.cx, R.Lx, R.hx), dy0 = wrap_diff(r0.y - P.cy, R.Ly, R.hy);
    if (!in_pore(P.kind, P.r0, P.r1, P.r_cavity, P.width, dx0, dy0, r0.z, h)) continue;
    const double dx = wrap_diff(r.x - P.cx, R.Lx, R.hx), dy = wrap_diff(r.y - P.cy, R.Ly, R.hy);
    if (P.kind == 5) {
      if (dx >= P.r0) {
        r.x += 2.0 * (P.r0 - dx);
        v.x = -v.x;
      } else if (dx <= -P.r0) {
        r.x += 2.0 * (-P.r0 - dx);
        v.x = -v.x;
      }
      if (dy >= P.r1) {
        r.y += 2.0 * (P.r1 - dy);
        v.y = -v.y;
      } else if (dy <= -P.r1) {
        r.y += 2.0 * (-P.r1 - dy);
        v.y = -v.y;
      }
      const double fl = prism_floor(P.width, h);
      if (r.z <= fl) {
        r.z = 2.0 * fl - r.z;
        v.z = -v.z;
      }
    } else if (P.kind == 3) {
      const double hw = 0.5 * P.width;
      if (dy >= hw) {
        r.y += 2.0 * (hw - dy);
        v.y = -v.y;
      } else if (dy <= -hw) {
        r.y += 2.0 * (-hw - dy);
        v.y = -v.y;
      }
    }
    return;
  }
}

// ------------------------------------------------------------------------------------------------
// The end of a step and the start of the next: the second half-kick (Fig. 3) that the atomic forms
// owe, the Berendsen scaling (Fig. 4) owed by a thermostat step, and the next first half-kick and
// drift (Fig. 2). The step kernel pays what is owed on its way through; the settle kernels below pay
// it before anything outside a step reads velocities. Both routes share these helpers (the same
// arithmetic in the same order), so they give bit-identical velocities.
__device__ __forceinline__ void kick_v(dvec4& v, const dvec4& f, double h) {
  v.x += h * f.x;
  v.y += h * f.y;
  v.z += h * f.z;
}

__device__ __forceinline__ double vsq(const dvec4& v) { return v.x * v.x + v.y * v.y + v.z * v.z; }

// replica R rescales at the end of step s (Fig. 4: every n_th steps)
__device__ __forceinline__ bool thermo_due(const RepDev& R, long long s) {
  return s > 0 && R.n_th > 0 && R.n_vap > 0 && (s % R.n_th) == 0;
}

__device__ __forceinline__ long long thermo_owed(const Arrays& a) {
  return *reinterpret_cast<volatile const long long*>(a.thermo_owed);
}

// sum of |v(t+dt)|^2 over molecules [k0, k1) of replica R by the whole block (256 threads), with the
// owed half-kick applied on the fly: each thread adds its molecules in index order, the warps by a
// fixed butterfly, thread 0 the warps in order. Returns the sum in thread 0.
__device__ double thermo_chunk_sum(const Arrays& a, const RepDev& R, int k0, int k1, int pend) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    dvec4 v = a.vel[R.vap_off + k];
    if (pend) kick_v(v, a.frc[R.vap_off + k], R.half_dt_m);
    acc += vsq(v);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  __syncthreads();  // sh is free again
  return t;
}

// lambda of replica r (Fig. 4) from its chunk partial sums, by one warp: the lanes add chunks
// lane, lane + 32, ... and a fixed butterfly combines them. 1 when the replica is not due.
__device__ void thermo_lambda_warp(const Arrays& a, const PotDev& p, int r, long long owed) {
  const int lane = threadIdx.x & 31;
  const RepDev& R = a.reps[r];
  if (!thermo_due(R, owed)) {
    if (lane == 0) a.lambda[r] = 1.0;
    return;
  }
  const int nch = (R.n_vap + 1023) / 1024;
  double t = 0.0;
  for (int ch = lane; ch < nch; ch += 32) t += __ldcg(&a.rep_part[((size_t)r * a.rep_chunks + ch) * 8]);
  t = warp_sum(t);
  if (lane == 0) {
    const double T = p.mass * t / ((double)R.dims * (double)R.n_vap);
    double lam = 1.0;
    if (T > 0.0) lam = sqrt(1.0 + R.lam_coef * (R.T0 / T - 1.0));
    a.lambda[r] = lam;
    *a.any_scale = 1;
  }
}

constexpr long long kSpinLimit = 1ll << 22;  // polls of a grid-barrier wait (~0.5 s) before giving up

// Grid barrier of the step kernels (co-resident grids only): every block arrives once its work is
// written; on a step that owes a thermostat (owed != 0) the last to arrive turns the partial sums
// into lambda for every replica, and then releases the others. A generation barrier: a block
// reads the release generation, then arrives; the block whose arrival completes the count resets
// the count to zero and advances the generation, which every other block waits to see change. So
// any grid size works, launch after launch (a context's kernels may differ in grid). A wait is
// bounded: after kSpinLimit polls the block sets the sticky timeout status and gives up (the count
// is then left off zero: a context that reported MD_ETIMEOUT must be destroyed). Returns whether
// the block may go on.
__device__ bool thermo_barrier(const Arrays& a, const PotDev& p, long long owed) {
  __shared__ int s_last, s_ok;
  __syncthreads();  // the block's partial sums are written
  if (threadIdx.x == 0) {
    const unsigned long long gen = *reinterpret_cast<volatile unsigned long long*>(a.bar_release);
    __threadfence();
    const unsigned long long old = atomicAdd(a.bar_arrive, 1ull);
    s_last = old == gridDim.x - 1ull;
    s_ok = 1;
    if (!s_last) {
      long long spins = 0;
      while (*reinterpret_cast<volatile unsigned long long*>(a.bar_release) == gen) {
        if (++spins > kSpinLimit) {
          atomicOr(a.status, kStatusTimeout);
          s_ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (s_last) {
    if (owed)
      for (int r = threadIdx.x >> 5; r < a.n_reps; r += blockDim.x >> 5)
        thermo_lambda_warp(a, p, r, owed);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(a.bar_arrive, 0ull);  // the next barrier counts from zero
      __threadfence();
      atomicAdd(a.bar_release, 1ull);  // the others go on
    }
  }
  __syncthreads();  // (s_ok and s_last are read again only after the next barrier's first sync)
  return s_ok != 0;
}

// A check of the bounded wait: every block but the last arrives at the barrier; the last never
// does, so the others' waits run out after kSpinLimit polls and raise the timeout status -- the
// failure a lost block would cause, made on purpose, with nothing left waiting.
__global__ void k_barrier_check(Arrays a, PotDev p) {
  count_launch(a);
  if (blockIdx.x == gridDim.x - 1) return;  // the arrival that never comes
  thermo_barrier(a, p, 0);
}

// One molecule's part of a step's start: the owed second half-kick and, after a thermostat step of
// its replica, the Berendsen scaling (lambda from the grid barrier), then Fig. 2's half-kick and
// drift, the reflections, the x/y wrap and the instability test; the FP32 offsets or absolute
// FP32 position the step's pair kernel screens with. Returns the squared displacement since the
// molecule's position at the last list build (0 when it left the box, and in the small-system
// kernel, which keeps no lists). xin / xout: the positions read and written (the same array but in
// the small-system kernel, which alternates two).
constexpr int kIntAbsolute = 8;  // also the absolute FP32 position (small-system kernel)

__device__ __forceinline__ double advance_molecule(const Arrays& a, int i, int pend,
                                                   long long owed, int flags,
                                                   const dvec4* __restrict__ xin, dvec4* xout,
                                                   float4* xfout) {
  // (with one replica its record loads beside the molecule's own words, not after its index)
  const int my_rep = a.n_reps == 1 ? 0 : a.rep[i];
  const RepDev& R = a.reps[my_rep];
  dvec4 x = xin[i], v = a.vel[i];
  const dvec4 x_old = x;
  const dvec4 f = a.frc[i];
  if (owed) {
    // the end of a thermostat step (for some replica): the owed kick, the scaling, then this
    // step's half-kick -- as the settle kernels would do it, then this kernel
    if (pend) kick_v(v, f, R.half_dt_m);
    if (thermo_due(R, owed)) {
      const double lam = __ldcg(&a.lambda[my_rep]);
      v.x *= lam;
      v.y *= lam;
      v.z *= lam;
    }
    kick_v(v, f, R.half_dt_m);
  } else {
    // Fig. 2's half-kick; with a deferred second half-kick of the previous step (Fig. 3, same
    // force) owed, both at once
    kick_v(v, f, pend ? R.dt_m : R.half_dt_m);
  }
  x.x += R.dt * v.x;
  x.y += R.dt * v.y;
  x.z += R.dt * v.z;
  // the boundary tests compare bit patterns (integer instructions; the FP64 pipe does only the
  // arithmetic, and the adds behind the tests run only where a molecule crosses)
  if (gt_pos(x.z, R.hz)) {
    x.z = R.Lz - x.z;
    v.z = -v.z;
  } else if (gt_pos(neg_bits(x.z), R.hz)) {
    x.z = -R.Lz - x.z;
    v.z = -v.z;
  }
  if (R.hard) reflect_solid(a, R, x_old, x, v);
  if (ge_pos(x.x, R.hx)) x.x -= R.Lx;
  else if (gt_pos(neg_bits(x.x), R.hx)) x.x += R.Lx;
  if (ge_pos(x.y, R.hy)) x.y -= R.Ly;
  else if (gt_pos(neg_bits(x.y), R.hy)) x.y += R.Ly;
  const bool bad = !(abs_le(x.x, R.hx) && abs_le(x.y, R.hy) && abs_le(x.z, R.hz));
  if (bad) atomicOr(a.status, kStatusUnstable);
  xout[i] = x;
  a.vel[i] = v;
  if (flags & kIntZeroForces) a.frc[i] = make_dvec4(0.0, 0.0, 0.0, 0.0);
  if (flags & kIntAbsolute) {  // the small-system kernel: no lists, no skin check
    xfout[i] = make_float4(narrow_f64(x.x), narrow_f64(x.y), narrow_f64(x.z), 0.f);
    return 0.0;
  }
  // the FP32 offset from the home cell's centre (periodic in x and y); the displacement since the
  // last build is its change, both offsets taken from the same centre: FP32 work, no FP64
  float4 hi;
  if (flags & kIntLocalOffsetsLo) {
    float4 lo;
    local_offset_df(a, R, x, a.home[i], hi, lo);
    a.lpos_lo[i] = lo;
  } else {
    hi = local_offset(a, R, x, a.home[i]);
  }
  if (flags & (kIntLocalOffsets | kIntLocalOffsetsLo)) a.lpos[i] = hi;
  const float4 r0 = a.lref[i];
  const float dx = hi.x - r0.x, dy = hi.y - r0.y, dz = hi.z - r0.z;
  return bad ? 0.0 : widen_f32(dx * dx + dy * dy + dz * dz);
}

// Fig. 2: v(t+dt/2) = v + a dt/2 ; r(t+dt) = r + v(t+dt/2) dt  (the same r(t+dt) as r + v dt + a dt^2/2)
// The first kernel of every step, on a grid of co-resident blocks that walk the molecules with a
// stride. It pays what the previous step left owed, in this order per molecule: the deferred second
// half-kick (Fig. 3) v += (dt/2m) f, then -- when that step was a thermostat step of the molecule's
// replica -- the Berendsen scaling v *= lambda (Fig. 4); then this step's half-kick, drift,
// reflections, wrap and skin check. lambda needs the replica's sum of v(t+dt)^2 over all of its
// molecules: on such steps (one in n_th) every block first adds its share in fixed (replica, chunk
// of 1024 molecules) units and meets the others at thermo_barrier. The last block to finish decides
// this step's rebuild branch of the captured graph and whether the step owes a thermostat.
template <bool MIXED>
__global__ void __launch_bounds__(256, 4) k_integrate_first(Arrays a, PotDev p, StepConds sc,
                                                            int flags) {
  count_launch(a);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.step += 1;
    *a.any_scale = 0;
  }
  // the words this launch branches on, loaded together (one round trip to memory for all three)
  const int st = halted(a) ? 1 : 0;
  const int pend = *reinterpret_cast<volatile const int32_t*>(a.kick_pending);
  // the same value in every block: the last block of the previous launch wrote it
  const long long owed = thermo_owed(a);
  // uniform within the block (the partial sums below synchronise the block); another block of this
  // launch may raise a status bit meanwhile, so blocks can differ, but every block arrives at the
  // barrier whatever it reads here
  bool halt = __syncthreads_or(st) != 0;
  if (owed) {
    const int units = a.n_reps * a.rep_chunks;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {  // block-uniform
      const int r = u / a.rep_chunks, ch = u % a.rep_chunks;
      const RepDev& R = a.reps[r];
      if (halt || !thermo_due(R, owed) || ch * 1024 >= R.n_vap) continue;
      const double t = thermo_chunk_sum(a, R, ch * 1024, min(R.n_vap, ch * 1024 + 1024), pend);
      if (threadIdx.x == 0) a.rep_part[(size_t)u * 8] = t;
    }
    if (!thermo_barrier(a, p, owed)) halt = true;
  }
  int trig = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; !halt && i < a.n_total; i += stride) {
    const double d2 = advance_molecule(a, i, pend, owed, flags, a.pos, a.pos, a.xf);
    // a molecule at or beyond skin/2 from its position at the last build triggers a rebuild;
    // molecules below the grouping threshold (nearly all) issue no atomic at all
    if (ge_pos(d2, p.group_disp2))  // rare: only molecules well into their skin
      atomicMax(&a.rep_disp2[a.rep[i]], (unsigned long long)__double_as_longlong(d2));
    trig |= ge_pos(d2, p.half_skin2) ? 1 : 0;
  }
  if (__syncthreads_or(trig) && threadIdx.x == 0) atomicExch(a.force_rebuild, 1);
  // the last block to finish decides this step's rebuild branch (graph) and the thermostat it owes
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(a.blk_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // every word the decision needs, loaded together: the step, the status and the rebuild flag
  // (every other block raised it, if at all, before its fence and its count above)
  const long long s = *reinterpret_cast<volatile long long*>(a.step);
  bool stop = false, rb = false;
  if (threadIdx.x == 0) {
    stop = halted(a);
    rb = *reinterpret_cast<volatile const int32_t*>(a.force_rebuild) != 0;
  }
  int th = 0;
  for (int r = threadIdx.x; r < a.n_reps; r += blockDim.x)
    if (thermo_due(a.reps[r], s)) th = 1;
  th = __syncthreads_or(th);
  if (threadIdx.x == 0) {
    *a.blk_done = 0u;
    *a.thermo_owed = (!stop && th) ? s : 0ll;
    if (sc.use && sc.has_rebuild) cudaGraphSetConditional(sc.rebuild, (!stop && rb) ? 1u : 0u);
  }
}

// ------------------------------------------------------------------------------------------------
// Settling outside a step (before a state read, the observables or a state load): the owed
// half-kick (k_kick_pending, below the pair kernels), then the owed Berendsen scaling of Fig. 4 in
// three kernels -- sum v^2 per (replica, chunk of 1024 molecules), one warp per replica adds the
// chunks in order and sets lambda, every molecule is scaled -- with the same arithmetic as the step
// kernel's. The owed step is cleared afterwards (launch_settle).
__global__ void __launch_bounds__(256) k_thermo_partial(Arrays a) {
  count_launch(a);
  if (halted(a)) return;
  const int r = blockIdx.x / a.rep_chunks, ch = blockIdx.x % a.rep_chunks;
  const RepDev& R = a.reps[r];
  if (!thermo_due(R, thermo_owed(a))) return;
  const int k0 = ch * 1024, k1 = min(R.n_vap, k0 + 1024);
  const double t = thermo_chunk_sum(a, R, k0, k1, 0);  // the kick was settled before
  if (threadIdx.x == 0) a.rep_part[(size_t)blockIdx.x * 8] = t;
}

__global__ void k_thermo_lambda(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a)) return;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= a.n_reps) return;
  thermo_lambda_warp(a, p, r, thermo_owed(a));
}

__global__ void k_thermo_scale(Arrays a) {
  count_launch(a);
  if (halted(a) || *reinterpret_cast<volatile int*>(a.any_scale) == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  const double lam = a.lambda[a.rep[i]];
  if (lam == 1.0) return;
  dvec4 v = a.vel[i];
  v.x *= lam;
  v.y *= lam;
  v.z *= lam;
  a.vel[i] = v;
}

// ------------------------------------------------------------------------------------------------
// cell build: a counting sort of the vapour by cell, stable in the caller's molecule index

// cells of the replicas that rebuild start from zero counts. The occupied ones are exactly the
// home cells of their molecules at the last build (the rest are zero already), so the clear runs
// over molecules, not cells. The other replicas keep their counts, so the scan over every cell
// reproduces their starts.
__global__ void k_cell_clear(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *a.n_act = 0;
  if (i >= a.n_total || !rep_rebuilds(a, a.rep[i])) return;
  const RepDev& R = a.reps[a.rep[i]];
  const int h = a.home[i];
  const int ix = h & 1023, iy = (h >> 10) & 1023, iz = (h >> 20) & 1023;
  if (ix < R.ncx && iy < R.ncy && iz < R.ncz)
    a.vcount[R.cell_off + (iz * R.ncy + iy) * R.ncx + ix] = 0;
}

// the whole cell scan by one block (at most 16 x 4096 cells; k_scan_single runs it with 1024
// threads): each thread owns a contiguous
// segment of whole int4s, sums it, takes its exclusive offset from a block scan of the sums and
// writes its segment; every load is issued up front, one round trip to memory per pass
__device__ void cell_scan_block(const Arrays& a) {
  __shared__ int warp_tot[32];
  const int n = a.n_cells, t = threadIdx.x, nthr = blockDim.x;
  const int S = (((n + nthr - 1) / nthr) + 3) & ~3;
  const int b0 = min(t * S, n), b1 = min(b0 + S, n);
  const int* __restrict__ in = a.vcount;
  int sum = 0;
  for (int k = b0; k < b1; k += 4) {
    if (k + 3 < b1) {
      const int4 v = *reinterpret_cast<const int4*>(in + k);
      sum += v.x + v.y + v.z + v.w;
    } else {
      for (int u = k; u < b1; ++u) sum += in[u];
    }
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if ((t & 31) >= o) incl += y;
  }
  if ((t & 31) == 31) warp_tot[t >> 5] = incl;
  __syncthreads();
  if (t < 32) {
    const int w = t < (nthr >> 5) ? warp_tot[t] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, wi, o);
      if (t >= o) wi += y;
    }
    if (t < (nthr >> 5)) warp_tot[t] = wi - w;
  }
  __syncthreads();
  int run = warp_tot[t >> 5] + incl - sum;
  for (int k = b0; k < b1; k += 4) {
    if (k + 3 < b1) {
      const int4 v = *reinterpret_cast<const int4*>(in + k);
      int4 o;
      o.x = run;
      o.y = o.x + v.x;
      o.z = o.y + v.y;
      o.w = o.z + v.z;
      run = o.w + v.w;
      *reinterpret_cast<int4*>(a.vstart + k) = o;
    } else {
      for (int u = k; u < b1; ++u) {
        a.vstart[u] = run;
        run += in[u];
      }
    }
  }
  if (t == 0) a.vstart[n] = a.n_total;
}

// Each molecule of a rebuilding replica takes its cell and a slot in it, and stages its record in
// the alternate arrays (same index), from which k_permute writes it to its sorted place. A cell's
// first molecule lists it among the active cells; the list grows by one atomic per warp (a single
// shared counter would otherwise see one atomic per occupied cell).
__global__ void k_cell_count(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool own = i < a.n_total && rep_rebuilds(a, a.rep[i]);
  int c = 0, ix = 0, iy = 0, iz = 0;
  bool first = false;
  if (own) {
    const RepDev& R = a.reps[a.rep[i]];
    const dvec4 x = a.pos[i];
    // (a multiplication by the inverse side, not an FP64 division: a molecule a rounding error
    // outside its cell stays far inside the margin the early skin check leaves)
    ix = cell_coord_mul(x.x, R.hx, R.ilcx, R.ncx);
    iy = cell_coord_mul(x.y, R.hy, R.ilcy, R.ncy);
    iz = cell_coord_mul(x.z, R.hz, R.ilcz, R.ncz);
    c = R.cell_off + (iz * R.ncy + iy) * R.ncx + ix;
    a.cell_tmp[i] = c;
    const int slot = atomicAdd(&a.vcount[c], 1);
    a.slot_tmp[i] = slot;
    first = slot == 0;
    a.pos_alt[i] = x;
    a.vel_alt[i] = a.vel[i];
    a.frc_alt[i] = a.frc[i];
    a.id_alt[i] = a.id[i];
  }
  const unsigned fm = __ballot_sync(kFull, first);
  if (fm) {
    const int lane = threadIdx.x & 31, leader = __ffs(fm) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(a.n_act, __popc(fm));
    base = __shfl_sync(kFull, base, leader);
    if (first) {
      const int k = base + __popc(fm & ((1u << lane) - 1u));
      a.act_cells[k] = c;
      a.act_rep[k] = a.rep[i];
      a.act_home[k] = pack_home(ix, iy, iz);
    }
  }
}

// exclusive scan of a 4096-element tile by 1024 threads; returns the tile total
__device__ int tile_exclusive_scan(const int32_t* in, int32_t* out, int n, int base) {
  __shared__ int warp_tot[32];
  __shared__ int total;
  const int t = threadIdx.x;
  int v[4];
  int run = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int idx = base + 4 * t + k;
    v[k] = idx < n ? in[idx] : 0;
    run += v[k];
  }
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if ((t & 31) >= o) incl += y;
  }
  if ((t & 31) == 31) warp_tot[t >> 5] = incl;
  __syncthreads();
  if (t < 32) {
    const int w = warp_tot[t];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, wi, o);
      if (t >= o) wi += y;
    }
    warp_tot[t] = wi - w;
  }
  __syncthreads();
  int ex = warp_tot[t >> 5] + incl - run;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int idx = base + 4 * t + k;
    if (idx < n) out[idx] = ex;
    ex += v[k];
  }
  if (t == 1023) total = ex;
  __syncthreads();
  const int r = total;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int tot = tile_exclusive_scan(a.vcount, a.vstart, a.n_cells, blockIdx.x * 4096);
  if (threadIdx.x == 0) a.scan_tiles[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(Arrays a, PotDev p, int ntiles) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  tile_exclusive_scan(a.scan_tiles, a.scan_tiles, ntiles, 0);
}

__global__ void __launch_bounds__(1024) k_scan_add(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int add = a.scan_tiles[blockIdx.x];
  for (int k = threadIdx.x; k < 4096; k += blockDim.x) {
    const int idx = blockIdx.x * 4096 + k;
    if (idx < a.n_cells) a.vstart[idx] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.vstart[a.n_cells] = a.n_total;
}

__global__ void __launch_bounds__(1024) k_scan_single(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  cell_scan_block(a);
}

__global__ void k_scatter(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total || !rep_rebuilds(a, a.rep[i])) return;
  a.perm_tmp[MD_CHK(a, a.vstart[MD_CHK(a, a.cell_tmp[i], a.n_cells)] + a.slot_tmp[i], a.n_total)] = i;
}

// within a cell, molecules are ordered by their caller index: the sorted order depends only on
// the positions, not on the order in which atomics were served. Records move from the staged copy
// (k_cell_count) to their sorted place.
__global__ void k_permute(Arrays a, PotDev p, int count_build) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  // the cell method has no list build, which counts the builds otherwise
  if (count_build && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.n_rebuilds, 1ull);
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_total || !rep_rebuilds(a, a.rep[s])) return;  // replicas occupy fixed ranges
  const int src = MD_CHK(a, a.perm_tmp[s], a.n_total);
  const int c = MD_CHK(a, a.cell_tmp[src], a.n_cells);
  const int my_id = a.id_alt[src];
  const int b = a.vstart[c], e = a.vstart[c + 1];
  int rank = 0;
  for (int t = b; t < e; ++t) rank += a.id_alt[MD_CHK(a, a.perm_tmp[t], a.n_total)] < my_id;
  const int dst = MD_CHK(a, b + rank, a.n_total);
  const dvec4 x = a.pos_alt[src];
  a.pos[dst] = x;
  a.vel[dst] = a.vel_alt[src];
  a.frc[dst] = a.frc_alt[src];
  a.id[dst] = my_id;
  const RepDev& R = a.reps[a.rep[src]];
  const int local = c - R.cell_off;
  const int ix = local % R.ncx, iy = (local / R.ncx) % R.ncy, iz = local / (R.ncx * R.ncy);
  const int home = pack_home(ix, iy, iz);
  a.home[dst] = home;
  float4 lhi, llo;
  local_offset_df(a, R, x, home, lhi, llo);
  a.lpos[dst] = lhi;
  a.lpos_lo[dst] = llo;
  a.lref[dst] = lhi;  // the skin check's reference
}

// ------------------------------------------------------------------------------------------------
// Verlet-list build, one warp per cell. The candidates of the 27 neighbour cells form a stream --
// first every vapour molecule of the 27 cells, then every wall atom -- and each lane holds one
// candidate of a 32-wide chunk; the cell's molecules are tested against the chunk one after another
// and hits are placed by ballot + prefix count, so lists are deterministic. A molecule i's list is
// one row of `cap` slots (row-major): partners j > i and then wall atoms fill it from the front,
// partners j < i from the back. The front is the FP64 half list (vapour partners first, so a
// vapour entry's slot is its pairbuf slot); front + back is the full list. Distances use the FP32
// cell-local offsets as (l_i - l_j) - dc*cell, which is exactly antisymmetric, so i lists j exactly
// when j lists i; the list radius carries a margin above the FP32 error.

// warp-aggregated update of a block's length histogram in shared memory (one shared atomic per
// distinct length in the warp); the block adds its nonzero counts to the global histogram once at
// the end -- a few hundred thousand cells adding to a few global bins one by one would queue on
// the same L2 addresses
__device__ __forceinline__ void hist_add(int* s_hist, int h, bool on) {
  const unsigned act = __ballot_sync(kFull, on);
  if (!on) return;
  const unsigned grp = __match_any_sync(act, h);
  if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&s_hist[h], __popc(grp));
}

// Processing order (optional). Molecules sorted by the length of the list the pair kernel walks
// (FP64: the front; mixed: front + back), longest first: warps see uniform lengths and the heaviest
// chunks start first. Whatever the order, each molecule's force is a sum it owns, so the order
// changes no result. The list build counts the lengths; its last block turns the counts into the
// start of each length, longest first (and clears them); k_order_assign places the molecules.
__device__ __forceinline__ int order_length(const Arrays& a, const PotDev& p, int i, int half) {
  return min(half ? a.n_front[i] : a.n_front[i] + a.n_back[i], p.cap);
}

// exclusive scan of the length histogram in descending order of length, by one whole block
__device__ void order_scan_block(const Arrays& a, const PotDev& p) {
  __shared__ int warp_tot[32];
  const int t = threadIdx.x, nthr = blockDim.x;
  const int per = (p.cap + nthr) / nthr;  // lengths cap .. 0 (cap + 1 of them), `per` a thread
  int sum = 0;
  for (int k = 0; k < per; ++k) {
    const int b = p.cap - (t * per + k);
    if (b >= 0) sum += a.hist[b];
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if ((t & 31) >= o) incl += y;
  }
  if ((t & 31) == 31) warp_tot[t >> 5] = incl;
  __syncthreads();
  if (t < 32) {
    const int w = t < (nthr >> 5) ? warp_tot[t] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, wi, o);
      if (t >= o) wi += y;
    }
    if (t < (nthr >> 5)) warp_tot[t] = wi - w;
  }
  __syncthreads();
  int run = warp_tot[t >> 5] + incl - sum;
  for (int k = 0; k < per; ++k) {
    const int b = p.cap - (t * per + k);
    if (b >= 0) {
      const int v = a.hist[b];
      a.hstart[b] = run;
      run += v;
      a.hist[b] = 0;
    }
  }
}

// Which list build runs: mode 0 lets the device choose -- a thread per molecule when the
// rebuilding replicas hold at least 65,536 molecules at under 2.5 per occupied cell (dilute vapour,
// where a warp per cell idles through cells of one molecule; fewer molecules leave too few
// threads to hide each one's serial walk), else a warp per cell; mode 1 forces the warp per cell,
// mode 2 the thread per molecule. Both build kernels are launched and read the same device
// values; the one not chosen returns at once.
__device__ __forceinline__ bool molecule_build(const Arrays& a, int mode) {
  if (mode != 0) return mode == 2;
  long long nm = 0;
  for (int r = 0; r < a.n_reps; ++r)
    if (rep_rebuilds(a, r)) nm += a.reps[r].n_vap;
  const long long na = *reinterpret_cast<volatile const int32_t*>(a.n_act);
  return nm >= 65536 && 2 * nm < 5 * na;
}

// the end of either list build, by every thread of a block: the block's longest row into max_nb,
// and with a processing order its length counts into the global histogram; the last block to
// finish turns the counts into the start of each length
__device__ void list_build_finish(const Arrays& a, const PotDev& p, int order, const int* s_hist,
                                  int s_max, int* s_last) {
  __syncthreads();
  if (threadIdx.x == 0 && s_max) atomicMax(a.max_nb, s_max);
  if (!order) return;
  for (int b = threadIdx.x; b <= p.cap; b += blockDim.x)
    if (s_hist[b]) atomicAdd(&a.hist[b], s_hist[b]);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    *s_last = atomicAdd(a.chain_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  order_scan_block(a, p);
  if (threadIdx.x == 0) *a.chain_done = 0u;
}

// Verlet-list build, one thread per molecule, for dilute vapour. Each thread walks its home cell's
// 27 neighbours in the warp build's order -- every vapour molecule of the 27 cells, then every wall
// atom -- testing each candidate against its FP32 offset as the warp build does, and writes its own
// row: the same entries in the same slots (front from the start, back from the end, in candidate
// order), so either build gives the same lists. Candidates are loaded four at a time.
constexpr int kListThreads = 128;

__global__ void __launch_bounds__(kListThreads) k_list_build_mol(Arrays a, PotDev p, int half,
                                                                 int front_only, int order,
                                                                 int mode) {
  count_launch(a);
  if (!need_rebuild(a, p)) return;  // (the flag holds still while the chain runs)
  __shared__ int s_run, s_last, s_max, s_go;
  __shared__ int s_hist[kMaxCap + 1];
  if (threadIdx.x == 0) s_go = molecule_build(a, mode);
  __syncthreads();
  if (!s_go) return;  // the warp build runs (uniform: every block reads the same values)
  if (threadIdx.x == 0) {
    s_run = !halted(a);
    s_max = 0;
  }
  if (order)
    for (int b = threadIdx.x; b <= p.cap; b += blockDim.x) s_hist[b] = 0;
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.n_rebuilds, 1ull);
  const int N = a.n_total, cap = p.cap;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int len = 0;
  bool counted = false;
  if (s_run && i < N) {
    const int r = a.rep[i];
    if (!rep_rebuilds(a, r)) {  // a kept row counts towards the processing order as it is
      len = order_length(a, p, i, half);
      counted = true;
    } else {
      const RepDev& R = a.reps[r];
      const int home = a.home[i];
      const int ix = home & 1023, iy = (home >> 10) & 1023, iz = (home >> 20) & 1023;
      const int c = R.cell_off + (iz * R.ncy + iy) * R.ncx + ix;
      const float4 li = a.lpos[i];
      uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      int nf = 0, nb = 0, nvh = 0;
      for (int pass = 0; pass < 2; ++pass) {
        const bool wallpass = pass == 1;
        for (int l = 0; l < 27; ++l) {
          const int dz = l / 9 - 1, dy = (l / 3) % 3 - 1, dx = l % 3 - 1;
          const int jz = iz + dz;
          if (jz < 0 || jz >= R.ncz) continue;
          int jy = iy + dy, jx = ix + dx;  // periodic in x and y
          jy += jy < 0 ? R.ncy : (jy >= R.ncy ? -R.ncy : 0);
          jx += jx < 0 ? R.ncx : (jx >= R.ncx ? -R.ncx : 0);
          const int cn = R.cell_off + (jz * R.ncy + jy) * R.ncx + jx;
          // half rows: a lower cell holds only lower molecule indices, no partner of a front
          if (!wallpass && front_only && cn < c) continue;
          const int k0 = wallpass ? a.wstart[cn] : a.vstart[cn];
          const int k1 = wallpass ? a.wstart[cn + 1] : a.vstart[cn + 1];
          const uint32_t code =
              ((uint32_t)(dx + 1) << 26) | ((uint32_t)(dy + 1) << 28) | ((uint32_t)(dz + 1) << 30);
          const float ox = cell_shift((uint32_t)(dx + 1), R.lcxf);
          const float oy = cell_shift((uint32_t)(dy + 1), R.lcyf);
          const float oz = cell_shift((uint32_t)(dz + 1), R.lczf);
          for (int k = k0; k < k1; k += 4) {
            float4 b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int kk = k + u < k1 ? k + u : k;
              b[u] = wallpass ? a.wlpos[MD_CHK(a, kk, a.n_wall_total)] : a.lpos[MD_CHK(a, kk, N)];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = k + u;
              if (j >= k1) break;
              const float ddx = (li.x - b[u].x) - ox, ddy = (li.y - b[u].y) - oy,
                          ddz = (li.z - b[u].z) - oz;
              const bool hit = (wallpass || j != i) && ddx * ddx + ddy * ddy + ddz * ddz < p.rl2f;
              if (!hit) continue;
              const uint32_t entry = (uint32_t)(wallpass ? N + j : j) | code;
              if (wallpass || j > i) {  // front, from the row's start
                if (nf < cap) row[nf] = entry;
                ++nf;
              } else if (!front_only) {  // back, from the row's end
                if (cap - 1 - nb >= 0) row[cap - 1 - nb] = entry;
                ++nb;
              }
            }
          }
        }
        if (!wallpass) nvh = nf;
      }
      const int nfc = min(nf, cap), nbc = min(nb, cap - nfc);
      if (nf + nb > cap || (half && (nvh > p.cap_v || nb > p.cap_v)))
        atomicOr(a.status, kStatusOverflow);
      a.n_front[i] = nfc;
      a.n_back[i] = nbc;
      a.n_vh[i] = min(nvh, p.cap_v);
      len = min(half ? nfc : nfc + nbc, cap);
      counted = true;
      atomicMax(&s_max, nf + nb);
    }
  }
  if (order) hist_add(s_hist, len, counted);
  list_build_finish(a, p, order, s_hist, s_max, &s_last);
}

// lane l < 27 of a list-build warp: the vapour and wall ranges of neighbour cell l of cell c
// (replica r, coordinates packed in home) -- (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1), periodic in x and y, none beyond z -- with
// no vapour for a lower cell in the half-row build (a lower cell holds only lower molecule
// indices in the cell-sorted order: no partner of a front). Empty ranges for c < 0 and lanes 27-31.
__device__ __forceinline__ void cell_ranges(const Arrays& a, int c, int r, int home, int front_only,
                                            int lane, int& vj0, int& nv, int& wj0, int& nw) {
  vj0 = nv = wj0 = nw = 0;
  if (c < 0 || lane >= 27) return;
  const RepDev& R = a.reps[r];
  const int ix = home & 1023, iy = (home >> 10) & 1023, iz = (home >> 20) & 1023;
  const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
  const int jz = iz + dz;
  if (jz < 0 || jz >= R.ncz) return;
  int jy = iy + dy, jx = ix + dx;  // periodic in x and y
  jy += jy < 0 ? R.ncy : (jy >= R.ncy ? -R.ncy : 0);
  jx += jx < 0 ? R.ncx : (jx >= R.ncx ? -R.ncx : 0);
  const int cn = R.cell_off + (jz * R.ncy + jy) * R.ncx + jx;
  vj0 = a.vstart[cn];
  nv = (front_only && cn < c) ? 0 : a.vstart[cn + 1] - vj0;
  wj0 = a.wstart[cn];
  nw = a.wstart[cn + 1] - wj0;
}

constexpr int kListWarps = 4;      // warps (cells) per block of the list build
constexpr int kStreamWin = 1024;   // candidate-stream window held in shared memory per warp

__global__ void __launch_bounds__(kListWarps * 32, 8) k_list_build(Arrays a, PotDev p, int half,
                                                                 int front_only, int order,
                                                                 int mode) {
  count_launch(a);
  if (!need_rebuild(a, p)) return;  // (the flag holds still while the chain runs)
  __shared__ uint32_t sh_stream[kListWarps][kStreamWin];
  __shared__ float4 sh_li[kListWarps][32];
  __shared__ int s_run, s_last, s_max, s_go;
  __shared__ int s_hist[kMaxCap + 1];  // this block's list-length counts (processing order)
  if (threadIdx.x == 0) s_go = !molecule_build(a, mode);
  __syncthreads();
  if (!s_go) return;  // the thread-per-molecule build runs (uniform in the block)
  // every block reports in at the end (the last one scans the length counts), so a block that
  // finds an error flag raised skips its work but not its report
  if (threadIdx.x == 0) {
    s_run = !halted(a);
    s_max = 0;
  }
  if (order)
    for (int b = threadIdx.x; b <= p.cap; b += blockDim.x) s_hist[b] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.n_rebuilds, 1ull);
  // a fixed grid; each warp takes the occupied cells of the rebuilding replicas in turn (the rows
  // it writes are its cell's molecules', so the order of the cells changes nothing)
  const int n_act = s_run ? *a.n_act : 0;
  // lane l < 27 stands for neighbour cell l = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); lane 13 is
  // the cell itself
  const uint32_t code =
      lane < 27 ? ((uint32_t)(lane % 3) << 26) | ((uint32_t)((lane / 3) % 3) << 28) |
                      ((uint32_t)(lane / 9) << 30)
                : 0u;
  // the cells come in a pipeline: the cell after next's index and replica, and the next cell's
  // neighbour ranges, load while this cell's candidates are screened
  const int stride = gridDim.x * kListWarps;
  int ac = blockIdx.x * kListWarps + w;
  int c_cur = -1, r_cur = 0, h_cur = 0, c_nxt = -1, r_nxt = 0, h_nxt = 0;
  if (ac < n_act) {
    c_cur = MD_CHK(a, a.act_cells[ac], a.n_cells);
    r_cur = a.act_rep[ac];
    h_cur = a.act_home[ac];
  }
  if (ac + stride < n_act) {
    c_nxt = MD_CHK(a, a.act_cells[ac + stride], a.n_cells);
    r_nxt = a.act_rep[ac + stride];
    h_nxt = a.act_home[ac + stride];
  }
  int vj0, nv, wj0, nw;
  cell_ranges(a, c_cur, r_cur, h_cur, front_only, lane, vj0, nv, wj0, nw);
  for (; c_cur >= 0; ac += stride) {
    const RepDev& R = a.reps[r_cur];
    int c_n2 = -1, r_n2 = 0, h_n2 = 0;
    if (ac + 2 * stride < n_act) {
      c_n2 = MD_CHK(a, a.act_cells[ac + 2 * stride], a.n_cells);
      r_n2 = a.act_rep[ac + 2 * stride];
      h_n2 = a.act_home[ac + 2 * stride];
    }
    int nvj0, nnv, nwj0, nnw;
    cell_ranges(a, c_nxt, r_nxt, h_nxt, front_only, lane, nvj0, nnv, nwj0, nnw);
    const int i_begin = __shfl_sync(kFull, vj0, 13), i_end = i_begin + __shfl_sync(kFull, nv, 13);
    const unsigned lt = (1u << lane) - 1u;
    const int N = a.n_total, cap = p.cap;
    uint32_t* stream = sh_stream[w];
    int max_n = 0;
    for (int ib = i_begin; ib < i_end; ib += 32) {
      const int nic = min(32, i_end - ib);
      // the molecules of this group: FP32 offsets in shared memory; lane il keeps molecule il's
      // front and back counts in registers
      sh_li[w][lane] = lane < nic ? a.lpos[ib + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      int cf = 0, cb = 0, vh = 0;
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass) {
        const bool wallpass = pass == 1;
        const int tot = wallpass ? nw : nv;
        const uint32_t base_idx = wallpass ? (uint32_t)(N + wj0) : (uint32_t)vj0;
        int incl = tot;
  #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int T = __shfl_sync(kFull, incl, 31);
        const int excl = incl - tot;
        for (int W0 = 0; W0 < T; W0 += kStreamWin) {
          const int W1 = min(T, W0 + kStreamWin);
          // lane l writes the part of its cell's candidates that falls in this window
          for (int m = max(0, W0 - excl); m < tot && excl + m < W1; ++m)
            stream[excl + m - W0] = (base_idx + (uint32_t)m) | code;
          __syncwarp();
          for (int base = W0; base < W1; base += 32) {
            const int q = base + lane;
            const bool valid = q < W1;
            const uint32_t entry = valid ? stream[q - W0] : 0u;
            const int jj = (int)(entry & kIndexMask);
            const int j = !valid ? 0 : wallpass ? MD_CHK(a, jj - N, a.n_wall_total) : MD_CHK(a, jj, N);
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) b = wallpass ? a.wlpos[j] : a.lpos[j];
            const float ox = cell_shift((entry >> 26) & 3u, R.lcxf);
            const float oy = cell_shift((entry >> 28) & 3u, R.lcyf);
            const float oz = cell_shift(entry >> 30, R.lczf);
            for (int il = 0; il < nic; ++il) {
              const int i = ib + il;
              const float4 li = sh_li[w][il];
              const float dx = (li.x - b.x) - ox, dy = (li.y - b.y) - oy, dz = (li.z - b.z) - oz;
              const bool hit = valid && (wallpass || j != i) && dx * dx + dy * dy + dz * dz < p.rl2f;
              const bool front = hit && (wallpass || j > i);
              const bool back = hit && !front && !front_only;
              const unsigned bf = __ballot_sync(kFull, front), bb = __ballot_sync(kFull, back);
              if (bf | bb) {
                const int f0 = __shfl_sync(kFull, cf, il), b0 = __shfl_sync(kFull, cb, il);
                if (front || back) {  // front from the row's start, back from its end, in stream order
                  const int slot = front ? f0 + __popc(bf & lt) : cap - 1 - (b0 + __popc(bb & lt));
                  if (front ? slot < cap : slot >= 0) a.nbr[(size_t)i * cap + slot] = entry;
                }
                if (lane == il) {
                  cf += __popc(bf);
                  cb += __popc(bb);
                }
              }
            }
          }
          __syncwarp();
        }
        if (!wallpass) vh = cf;
      }
      // counts, overflow, processing-order histogram
      {
        const int i = ib + lane;
        const bool own = lane < nic;
        const int nf = cf, nb = cb, nvh = vh;
        const int nfc = min(nf, cap), nbc = min(nb, cap - min(nf, cap));
        if (own) {
          if (nf + nb > cap || (half && (nvh > p.cap_v || nb > p.cap_v)))
            atomicOr(a.status, kStatusOverflow);
          a.n_front[i] = nfc;
          a.n_back[i] = nbc;
          a.n_vh[i] = min(nvh, p.cap_v);
          max_n = max(max_n, nf + nb);
        }
        if (order) hist_add(s_hist, min(half ? nfc : nfc + nbc, cap), own);
      }
      __syncwarp();
    }
  #pragma unroll
    for (int o = 16; o; o >>= 1) max_n = max(max_n, __shfl_xor_sync(kFull, max_n, o));
    if (lane == 0 && max_n) atomicMax(&s_max, max_n);  // (the block's, added once at the end)
    c_cur = c_nxt;
    r_cur = r_nxt;
    h_cur = h_nxt;
    c_nxt = c_n2;
    r_nxt = r_n2;
    h_nxt = h_n2;
    vj0 = nvj0;
    nv = nnv;
    wj0 = nwj0;
    nw = nnw;
  }
  // the kept rows of the replicas that do not rebuild count too
  if (order && s_run) {
    const int nw = gridDim.x * kListWarps;
    for (int base = (blockIdx.x * kListWarps + w) * 32; base < a.n_total; base += nw * 32) {
      const int i = base + lane;
      const bool own = i < a.n_total && !rep_rebuilds(a, a.rep[i]);
      hist_add(s_hist, own ? order_length(a, p, i, half) : 0, own);
    }
  }
  list_build_finish(a, p, order, s_hist, s_max, &s_last);
}

// ------------------------------------------------------------------------------------------------
// processing position of each molecule (warp-aggregated atomics on the length starts)
__global__ void k_order_assign(Arrays a, PotDev p, int half) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool own = i < a.n_total;
  const int h = own ? order_length(a, p, i, half) : 0;
  const unsigned act = __ballot_sync(kFull, own);
  if (!own) return;
  const unsigned grp = __match_any_sync(act, h);
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if ((threadIdx.x & 31) == leader) base = atomicAdd(&a.hstart[h], __popc(grp));
  base = __shfl_sync(grp, base, leader);
  const int pos = base + __popc(grp & ((1u << (threadIdx.x & 31)) - 1u));
  if (pos < a.n_total) a.order[pos] = i;
}

// FP64: for each vapour pair (i, j > i) at front slot k of i, find i in j's back region (slot m)
// and record fwd[i, k] = j * cap_v + m: the half-list pass stores the pair force where j's gather
// reads it, in j's own list order. Every back slot is the target of exactly one pair, so the gather
// is deterministic and needs no atomics; a pair whose partner slot cannot be found (an overflowed
// list, already flagged) points at the spare entry past the end of pairbuf.
// One warp per molecule (grid-stride), lanes over the front slots; when the row length is a
// multiple of 4 the back region is scanned four entries per 16-byte load.
__global__ void __launch_bounds__(256) k_fwd_build(Arrays a, PotDev p) {
  count_launch(a);
  if (halted(a) || !need_rebuild(a, p)) return;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int cap = p.cap, capv = p.cap_v;
  const uint32_t spare = (uint32_t)((size_t)a.n_total * capv);
  const bool vec = (cap & 3) == 0;
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < a.n_total; i += warps) {
    if (!rep_rebuilds(a, a.rep[i])) continue;  // (warp-uniform: one molecule per warp)
    const int nvh = a.n_vh[i];
    const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
    uint32_t* __restrict__ fw = a.fwd + (size_t)i * capv;
    for (int k = threadIdx.x & 31; k < nvh; k += 32) {
      const uint32_t j = MD_CHK(a, row[k] & kIndexMask, a.n_total);
      const int nb = min(a.n_back[j], capv);
      const uint32_t* __restrict__ rj = a.nbr + (size_t)j * cap + cap;  // one past j's row
      int m = -1;
      if (vec) {
        // entries cap-4q-4 .. cap-4q-1 hold back slots 4q+3 .. 4q; 4q < nb <= cap keeps the load
        // inside row j
        const uint4* __restrict__ r4 = reinterpret_cast<const uint4*>(rj);
        for (int q = 0; 4 * q < nb; ++q) {
          const uint4 e = r4[-1 - q];
          if ((e.w & kIndexMask) == (uint32_t)i) { m = 4 * q; break; }
          if ((e.z & kIndexMask) == (uint32_t)i) { m = 4 * q + 1; break; }
          if ((e.y & kIndexMask) == (uint32_t)i) { m = 4 * q + 2; break; }
          if ((e.x & kIndexMask) == (uint32_t)i) { m = 4 * q + 3; break; }
        }
      } else {
        for (int q = 0; q < nb; ++q)
          if ((rj[-1 - q] & kIndexMask) == (uint32_t)i) { m = q; break; }
      }
      if (m < 0 || m >= nb) {
        atomicOr(a.status, kStatusOverflow);
        fw[k] = spare;
      } else {
        fw[k] = j * (uint32_t)capv + (uint32_t)m;
      }
    }
  }
}

// Warp-level dynamic work distribution over chunks of MPW molecules of the processing order.
// Returns the chunk (or -1 when the work is exhausted). The counters are reset by the last block.
template <int MPW>
__device__ __forceinline__ int next_chunk(const Arrays& a) {
  int c = 0;
  if ((threadIdx.x & 31) == 0) c = atomicAdd(a.work, 1);
  c = __shfl_sync(kFull, c, 0);
  return c * MPW < a.n_total ? c : -1;
}

// The chunks of a warp, in one of two walks. Dynamic (stat 0): each chunk from the work counter,
// so the longest-first chunks go to whichever warp is free. Static (stat 1): warp w takes chunks
// w, w + W, w + 2W, ... of the length-ordered molecules (W warps in the grid) -- no atomic per
// chunk -- and the next chunk's molecule index (its place in the processing order) is loaded while
// this chunk runs, taking two round trips to memory off each chunk's chain of dependent loads.
template <int MPW, int TPP>
struct ChunkWalk {
  int chunk, nw, ip;
  __device__ __forceinline__ int molecule(const Arrays& a, int t, int lpt) const {
    return lpt ? MD_CHK(a, a.order[t], a.n_total) : t;
  }
  __device__ __forceinline__ void start(const Arrays& a, int stat, int lpt) {
    const int lane = threadIdx.x & 31;
    nw = gridDim.x * (blockDim.x >> 5);
    chunk = stat ? blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) : next_chunk<MPW>(a);
    if (stat && chunk * MPW >= a.n_total) chunk = -1;
    const int t = chunk >= 0 ? chunk * MPW + lane / TPP : a.n_total;
    ip = stat && t < a.n_total ? molecule(a, t, lpt) : 0;
  }
  // the molecule of this lane in the current chunk (t < n_total), and the next chunk prefetched
  __device__ __forceinline__ int take(const Arrays& a, int stat, int lpt, int t) {
    if (!stat) return t < a.n_total ? molecule(a, t, lpt) : 0;
    const int here = ip;
    const int nxt = (chunk + nw) * MPW < a.n_total ? chunk + nw : -1;
    const int tn = nxt >= 0 ? nxt * MPW + (threadIdx.x & 31) / TPP : a.n_total;
    ip = tn < a.n_total ? molecule(a, tn, lpt) : 0;
    return here;
  }
  __device__ __forceinline__ void advance(const Arrays& a, int stat) {
    if (stat) chunk = (chunk + nw) * MPW < a.n_total ? chunk + nw : -1;
    else chunk = next_chunk<MPW>(a);
  }
};

// sum over the TPP lanes that share a molecule (fixed butterfly order: deterministic)
template <int TPP, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = TPP / 2; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int TPP>
__device__ __forceinline__ double group_min(double v) {
#pragma unroll
  for (int o = TPP / 2; o; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ void finish_chunks(const Arrays& a) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.work_done, 1u) == gridDim.x - 1) {
      *a.work = 0;
      *a.work_done = 0u;
    }
  }
}

// positive doubles compare like their bit patterns: an integer test, no FP64 instruction
__device__ __forceinline__ bool lt_pos(double x, double y) {
  return __double_as_longlong(x) < __double_as_longlong(y);
}

// ------------------------------------------------------------------------------------------------
// Pair forces (Eq. 2, Fig. 1): f_i = sum_j F(r_ij)/r_ij * (r_i - r_j) over pairs with r^2 < rc^2,
// F(r)/r = inv2 * inv6 * (48 eps s^12 inv6 - 24 eps s^6), inv2 = 1/r^2, inv6 = inv2^3.
// A warp takes chunks of 32/TPP molecules; the TPP lanes of a molecule split its list.
//
// FP64, half list: molecule i walks the front of its row; each vapour pair's force goes to the
// partner's back slot in pairbuf (fwd), where the partner's gather reads it in list order.

// One FP64 pair term: whether list entry e is within the cutoff of i and, if so, the force on i,
// p = F(r)/r * (r_i - r_j). The LJ part sits behind the cutoff branch: a warp whose lanes are all
// beyond the cutoff skips it, which a masked (branch-free) form cannot (measured: the masked
// two-entry form took ~9 % more FP64-pipe cycles).
// FP32 cell-local offset of list entry e's partner (a vapour molecule or a wall atom)
__device__ __forceinline__ float4 partner_lpos(const Arrays& a, uint32_t e, int N) {
  const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
  return j >= N ? a.wlpos[j - N] : a.lpos[j];
}

// position of list entry e's partner (a vapour molecule or a wall atom)
__device__ __forceinline__ dvec4 partner_pos(const Arrays& a, uint32_t e, int N) {
  const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
  return j >= N ? a.wpos[j - N] : a.pos[j];
}

__device__ __forceinline__ bool pair_term(const Arrays& a, const PotDev& p, const RepDev& R,
                                          const dvec4& xi, uint32_t e, const dvec4& xj, int N,
                                          double& px, double& py, double& pz) {
  const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
  const bool wall = j >= N;
  const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
  const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
  const double dz = xi.z - xj.z;
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (!lt_pos(r2, wall ? p.rcw2 : p.rc2)) return false;
  const double a12 = wall ? p.a12w : p.a12, b6 = wall ? p.b6w : p.b6;
  const double inv2 = rcp_nr(r2);
  const double inv6 = inv2 * inv2 * inv2;
  const double fr = inv2 * inv6 * fma(a12, inv6, -b6);
  px = fr * dx;
  py = fr * dy;
  pz = fr * dz;
  return true;
}

template <int TPP>
__global__ void __launch_bounds__(256) k_forces_half(Arrays a, PotDev p, int lpt) {
  constexpr int MPW = 32 / TPP;
  count_launch(a);
  clear_rebuild_flags(a);
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap, capv = p.cap_v;
  const int lane = threadIdx.x & 31, sub = lane & (TPP - 1);
  int cnt = 0;
  for (int chunk = next_chunk<MPW>(a); chunk >= 0; chunk = next_chunk<MPW>(a)) {
    const int t = chunk * MPW + lane / TPP;
    const bool live = t < N;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    int i = 0;
    if (live) {
      i = lpt ? MD_CHK(a, a.order[t], N) : t;
      const RepDev& R = a.reps[a.rep[i]];
      const dvec4 xi = a.pos[i];
      const int n = a.n_front[i], nvh = a.n_vh[i];
      const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      const uint32_t* __restrict__ fw = a.fwd + (size_t)i * capv;
      // software-pipelined: the next entry and its partner's position load while this pair's
      // FP64 chain runs
      uint32_t e = sub < n ? row[sub] : 0u;
      dvec4 xj = sub < n ? partner_pos(a, e, N) : xi;
      for (int k = sub; k < n; k += TPP) {
        const int kn = k + TPP;
        const uint32_t en = kn < n ? row[kn] : 0u;
        const dvec4 xn = kn < n ? partner_pos(a, en, N) : xi;
        double px = 0.0, py = 0.0, pz = 0.0;
        // warps whose lanes are all beyond the cutoff skip the pair term (a branch, not a mask)
        if (pair_term(a, p, R, xi, e, xj, N, px, py, pz)) {
          fx += px;
          fy += py;
          fz += pz;
          ++cnt;
        }
        if (k < nvh) a.pairbuf[MD_CHK(a, fw[k], (long long)a.n_total * p.cap_v + 1)] = make_dvec4(px, py, pz, 0.0);
        e = en;
        xj = xn;
      }
    }
    fx = group_sum<TPP>(fx);
    fy = group_sum<TPP>(fy);
    fz = group_sum<TPP>(fz);
    if (live && sub == 0) a.fpart[i] = make_dvec4(fx, fy, fz, 0.0);
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// FP64, half list, reaction forces by atomics: as k_forces_half, but each vapour pair's reaction
// goes straight to the partner's force with FP64 atomic adds (executed in L2, not on the SM's FP64
// pipe), and the molecule adds its own half-list sum the same way; no pair buffer, no gather. The
// forces must be zero beforehand. The order of the atomic adds varies from run to run, so the
// forces agree with the deterministic form to rounding, not bit for bit.
template <int TPP>
__global__ void __launch_bounds__(256) k_forces_half_atomic(Arrays a, PotDev p, int lpt,
                                                            int owe_kick, int stat) {
  constexpr int MPW = 32 / TPP;
  count_launch(a);
  clear_rebuild_flags(a);
  // in a step, the second half-kick is owed: the next first half-kick (or k_kick_pending) pays it
  if (owe_kick && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 1;
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap;
  const int lane = threadIdx.x & 31, sub = lane & (TPP - 1);
  int cnt = 0;
  ChunkWalk<MPW, TPP> walk;
  walk.start(a, stat, lpt);
  for (; walk.chunk >= 0; walk.advance(a, stat)) {
    const int chunk = walk.chunk;
    const int cnt0 = cnt;
    const int t = chunk * MPW + lane / TPP;
    const bool live = t < N;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    const int im = walk.take(a, stat, lpt, t);
    int i = 0;
    if (live) {
      i = im;
      const RepDev& R = a.reps[a.rep[i]];
      const dvec4 xi = a.pos[i];
      const int n = a.n_front[i], nvh = a.n_vh[i];
      const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      uint32_t e = sub < n ? row[sub] : 0u;
      dvec4 xj = sub < n ? partner_pos(a, e, N) : xi;
      for (int k = sub; k < n; k += TPP) {
        const int kn = k + TPP;
        const uint32_t en = kn < n ? row[kn] : 0u;
        const dvec4 xn = kn < n ? partner_pos(a, en, N) : xi;
        double px, py, pz;
        if (pair_term(a, p, R, xi, e, xj, N, px, py, pz)) {
          fx += px;
          fy += py;
          fz += pz;
          if (k < nvh) {  // Newton's third law: the partner receives -p
            const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
            atomicAdd(&a.frc[j].x, neg_bits(px));
            atomicAdd(&a.frc[j].y, neg_bits(py));
            atomicAdd(&a.frc[j].z, neg_bits(pz));
          }
          ++cnt;
        }
        e = en;
        xj = xn;
      }
    }
    fx = group_sum<TPP>(fx);
    fy = group_sum<TPP>(fy);
    fz = group_sum<TPP>(fz);
    // a molecule with no pair within the cutoff adds nothing (dilute vapour: about half of them)
    const int found = group_sum<TPP>(cnt - cnt0);
    if (live && sub == 0 && found) {
      atomicAdd(&a.frc[i].x, fx);
      atomicAdd(&a.frc[i].y, fy);
      atomicAdd(&a.frc[i].z, fz);
    }
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// FP64, half list, reaction forces by atomics, compacted: a warp takes kAqMols molecules, and the
// kAqLanes lanes of a molecule screen its list slots in FP32 on the cell-local offsets, kAqSub slots
// each at a time, keeping the entries that may lie within the cutoff (FP32 r^2 below
// rc^2 (1 + 1e-5); the FP32 error is ~1e-7 of rc^2) in a per-warp queue. When the queue is full
// enough, or the lists are done, the FP64 pair terms (the arithmetic of pair_term, the cutoff
// decided in FP64) run over the queue with every lane busy, two independent entries per lane; the
// reactions go to the partners by FP64 atomic adds; each pair's force is kept in shared memory, and
// every lane then sums the entries it queued, in slot order, before the molecule's lanes add their
// sums in a fixed order. A skin entry costs an FP32 screen instead of the FP64 difference and r^2,
// and no lane idles through another lane's pair term. Small chunks keep the warps balanced when a
// few molecules (those next to a wall) have rows several times longer than the rest.
constexpr int kAqLanes = 4;                  // lanes screening one molecule's row
constexpr int kAqMols = 32 / kAqLanes;       // molecules per warp chunk
constexpr int kAqSub = 4;                    // slots per lane screened at a time
constexpr int kAqCap = 256;                  // queue entries per warp
constexpr int kAqSeg = 4;                    // screened rounds held before a flush

struct AtomicQueue {
  double ox[kAqMols], oy[kAqMols], oz[kAqMols];  // FP64 positions of the warp's molecules
  double oLx[kAqMols], oLy[kAqMols];         // their replicas' box sides in x and y
  uint32_t othx[kAqMols], othy[kAqMols];     // and the high-word image thresholds
  uint32_t qe[kAqCap];                       // partner index | owner << 27
  double rx[kAqCap], ry[kAqCap], rz[kAqCap]; // pair force on the owner
};

// one queued FP64 pair term (slot u): the force on the owner kept in shared memory, the reaction
// sent to a vapour partner; returns whether the pair lies within the cutoff
__device__ __forceinline__ bool queued_term(const Arrays& a, const PotDev& p, AtomicQueue& S, int u,
                                            uint32_t q, const dvec4& xj, int N) {
  const int j = MD_CHK(a, (int)(q & kIndexMask), a.n_total + a.n_wall_total), m = (int)(q >> 27);
  const bool wall = j >= N;
  const double dx = image_hi(S.ox[m] - xj.x, S.oLx[m], S.othx[m]);
  const double dy = image_hi(S.oy[m] - xj.y, S.oLy[m], S.othy[m]);
  const double dz = S.oz[m] - xj.z;
  const double r2 = dx * dx + dy * dy + dz * dz;
  const bool in = lt_pos(r2, wall ? p.rcw2 : p.rc2);
  const double a12 = wall ? p.a12w : p.a12, b6 = wall ? p.b6w : p.b6;
  const double inv2 = rcp_nr(r2);
  const double inv6 = inv2 * inv2 * inv2;
  const double fr = in ? inv2 * inv6 * fma(a12, inv6, -b6) : 0.0;
  const double px = fr * dx, py = fr * dy, pz = fr * dz;
  S.rx[u] = px;
  S.ry[u] = py;
  S.rz[u] = pz;
  if (in && !wall) {  // Newton's third law: the partner receives -p
    atomicAdd(&a.frc[j].x, neg_bits(px));
    atomicAdd(&a.frc[j].y, neg_bits(py));
    atomicAdd(&a.frc[j].z, neg_bits(pz));
  }
  return in;
}

__device__ __forceinline__ dvec4 queued_partner(const Arrays& a, uint32_t q, int N) {
  const int j = MD_CHK(a, (int)(q & kIndexMask), a.n_total + a.n_wall_total);
  return j >= N ? a.wpos[j - N] : a.pos[j];
}

__global__ void __launch_bounds__(256) k_forces_atomic_packed(Arrays a, PotDev p, int lpt,
                                                              int owe_kick) {
  extern __shared__ __align__(32) unsigned char aq_smem[];
  AtomicQueue& S = reinterpret_cast<AtomicQueue*>(aq_smem)[threadIdx.x >> 5];
  count_launch(a);
  clear_rebuild_flags(a);
  if (owe_kick && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 1;
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap;
  const int lane = threadIdx.x & 31, sub = lane & (kAqLanes - 1), mol = lane / kAqLanes;
  int cnt = 0;
  for (int chunk = next_chunk<kAqMols>(a); chunk >= 0; chunk = next_chunk<kAqMols>(a)) {
    const int t = chunk * kAqMols + mol;
    const bool live = t < N;
    int i = 0, n = 0;
    float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
    float lcx = 0.f, lcy = 0.f, lcz = 0.f;
    if (live) {
      i = lpt ? MD_CHK(a, a.order[t], N) : t;
      n = a.n_front[i];
      li = a.lpos[i];
      const RepDev& R = a.reps[a.rep[i]];
      if (sub == 0) {
        const dvec4 xi = a.pos[i];
        S.ox[mol] = xi.x;
        S.oy[mol] = xi.y;
        S.oz[mol] = xi.z;
        S.oLx[mol] = R.Lx;
        S.oLy[mol] = R.Ly;
        S.othx[mol] = R.hi_thr_x;
        S.othy[mol] = R.hi_thr_y;
      }
      lcx = R.lcxf;
      lcy = R.lcyf;
      lcz = R.lczf;
    }
    const int nmax = __reduce_max_sync(kFull, n);
    const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    int Q = 0, nseg = 0;
    uint32_t seg[kAqSeg];  // the lane's queued runs: first entry | count << 16
#pragma unroll
    for (int g = 0; g < kAqSeg; ++g) seg[g] = 0u;
    for (int t0 = 0; t0 < nmax; t0 += kAqLanes * kAqSub) {
      // FP32 screen of the lane's slots t0 + k * kAqLanes + sub (entries, then partner offsets)
      uint32_t e[kAqSub];
#pragma unroll
      for (int k = 0; k < kAqSub; ++k) {
        const int sl = t0 + k * kAqLanes + sub;
        e[k] = sl < n ? row[sl] : 0u;
      }
      float4 b[kAqSub];
#pragma unroll
      for (int k = 0; k < kAqSub; ++k)
        b[k] = t0 + k * kAqLanes + sub < n ? partner_lpos(a, e[k], N) : li;
      unsigned hm = 0;
#pragma unroll
      for (int k = 0; k < kAqSub; ++k) {
        const bool wall = (int)(e[k] & kIndexMask) >= N;
        const float dx = (li.x - b[k].x) - cell_shift((e[k] >> 26) & 3u, lcx);
        const float dy = (li.y - b[k].y) - cell_shift((e[k] >> 28) & 3u, lcy);
        const float dz = (li.z - b[k].z) - cell_shift(e[k] >> 30, lcz);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (t0 + k * kAqLanes + sub < n && r2 < (wall ? p.rcw2f_hi : p.rc2f_hi)) hm |= 1u << k;
      }
      // append: the lane's survivors go to [Q + excl, Q + excl + c), in slot order
      const int c = __popc(hm);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      int w = Q + incl - c;
#pragma unroll
      for (int g = 0; g < kAqSeg; ++g)
        if (g == nseg) seg[g] = (uint32_t)w | ((uint32_t)c << 16);
#pragma unroll
      for (int k = 0; k < kAqSub; ++k)
        if ((hm >> k) & 1u) S.qe[w++] = (e[k] & kIndexMask) | ((uint32_t)mol << 27);
      Q += total;
      ++nseg;
      if (Q <= kAqCap - 32 * kAqSub && nseg < kAqSeg && t0 + kAqLanes * kAqSub < nmax) continue;
      __syncwarp();
      // FP64 pair terms over the queue, two entries per lane while at least 33 remain
      int u0 = 0;
      for (; u0 + 32 < Q; u0 += 64) {
        const int u1 = u0 + lane, u2 = u0 + 32 + lane;
        const bool v2 = u2 < Q;
        const uint32_t q1 = S.qe[u1], q2 = v2 ? S.qe[u2] : q1;
        const dvec4 x1 = queued_partner(a, q1, N);
        const dvec4 x2 = queued_partner(a, q2, N);
        cnt += queued_term(a, p, S, u1, q1, x1, N) ? 1 : 0;
        if (v2) cnt += queued_term(a, p, S, u2, q2, x2, N) ? 1 : 0;
      }
      if (u0 < Q && u0 + lane < Q) {
        const int u1 = u0 + lane;
        const uint32_t q1 = S.qe[u1];
        cnt += queued_term(a, p, S, u1, q1, queued_partner(a, q1, N), N) ? 1 : 0;
      }
      __syncwarp();
      // the entries this lane queued, in slot order
#pragma unroll
      for (int g = 0; g < kAqSeg; ++g) {
        if (g < nseg) {
          const int u_end = (int)(seg[g] & 0xffffu) + (int)(seg[g] >> 16);
          for (int u = (int)(seg[g] & 0xffffu); u < u_end; ++u) {
            fx += S.rx[u];
            fy += S.ry[u];
            fz += S.rz[u];
          }
        }
      }
      __syncwarp();
      Q = 0;
      nseg = 0;
    }
    fx = group_sum<kAqLanes>(fx);
    fy = group_sum<kAqLanes>(fy);
    fz = group_sum<kAqLanes>(fz);
    if (live && sub == 0 && n > 0) {
      atomicAdd(&a.frc[i].x, fx);
      atomicAdd(&a.frc[i].y, fy);
      atomicAdd(&a.frc[i].z, fz);
    }
    __syncwarp();
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// The owed second half-kick (Fig. 3), v(t+dt) = v(t+dt/2) + a(t+dt) dt/2, when the FP64 atomic form
// deferred it: applied before the thermostat, the observables or a state read. Every block reads
// the flag before its first thread reports in; the last block to report clears it.
__global__ void k_kick_pending(Arrays a, PotDev p) {
  count_launch(a);
  const int pend = *reinterpret_cast<volatile const int32_t*>(a.kick_pending);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (pend && !halted(a) && i < a.n_total) {
    const RepDev& R = a.reps[a.rep[i]];
    dvec4 v = a.vel[i];
    kick_v(v, a.frc[i], R.half_dt_m);
    a.vel[i] = v;
  }
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(a.kick_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *a.kick_pending = 0;
    *a.kick_done = 0u;
  }
}

__global__ void k_zero_forces(Arrays a) {
  count_launch(a);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n_total) a.frc[i] = make_dvec4(0.0, 0.0, 0.0, 0.0);
}

// FP64, every pair, no lists (the paper's F1 form, Fig. 1): one thread per molecule sums over every
// other vapour molecule and every wall atom of its replica, in index order. Pairs beyond the
// cutoff contribute nothing, so the pair set and the forces are those of the list path; the work
// is O(N^2) per replica (small systems). STATS computes the observable pass instead of forces.
template <bool STATS, bool KICK>
__global__ void __launch_bounds__(128) k_allpairs(Arrays a, PotDev p) {
  count_launch(a);
  if (!STATS) clear_rebuild_flags(a);
  if (KICK && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 0;  // this step kicks itself
  if (halted(a)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = a.n_total;
  const bool live = i < N;
  double fx = 0.0, fy = 0.0, fz = 0.0, pe = 0.0, vir = 0.0, pew = 0.0, virw = 0.0;
  double d2w = __longlong_as_double(0x7ff0000000000000ll);
  int cvv = 0, cvw = 0;
  if (live) {
    const RepDev& R = a.reps[a.rep[i]];
    const dvec4 xi = a.pos[i];
    for (int j = R.vap_off; j < R.vap_off + R.n_vap; ++j) {
      if (j == i) continue;
      const dvec4 xj = a.pos[j];
      const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
      const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
      const double dz = xi.z - xj.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!lt_pos(r2, p.rc2)) continue;
      const double inv2 = rcp_nr(r2), inv6 = inv2 * inv2 * inv2;
      const double fr = inv2 * inv6 * fma(p.a12, inv6, -p.b6);
      if (STATS) {
        pe += 0.5 * (inv6 * fma(p.e12, inv6, -p.e6) - p.ushift);
        vir += 0.5 * fr * r2;
      } else {
        fx = fma(fr, dx, fx);
        fy = fma(fr, dy, fy);
        fz = fma(fr, dz, fz);
      }
      ++cvv;
    }
    for (int w = R.wall_off; w < R.wall_off + R.n_wall; ++w) {
      const dvec4 xj = a.wpos[w];
      const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
      const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
      const double dz = xi.z - xj.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!lt_pos(r2, p.rcw2)) continue;
      const double inv2 = rcp_nr(r2), inv6 = inv2 * inv2 * inv2;
      const double fr = inv2 * inv6 * fma(p.a12w, inv6, -p.b6w);
      if (STATS) {
        pew += inv6 * fma(p.e12w, inv6, -p.e6w) - p.ushift_w;
        virw += fr * r2;
        d2w = fmin(d2w, r2);
      } else {
        fx = fma(fr, dx, fx);
        fy = fma(fr, dy, fy);
        fz = fma(fr, dz, fz);
      }
      ++cvw;
    }
    if (STATS) {
      a.pe_i[i] = pe;
      a.pevw_i[i] = pew;
      a.vir_i[i] = vir;
      a.virw_i[i] = virw;
      a.d2w_i[i] = d2w;
      a.cnt_vv_i[i] = cvv;
      a.cnt_vw_i[i] = cvw;
    } else {
      a.frc[i] = make_dvec4(fx, fy, fz, 0.0);
      if (KICK) {  // Fig. 3
        dvec4 v = a.vel[i];
        const double h = R.half_dt_m;
        v.x += h * fx;
        v.y += h * fy;
        v.z += h * fz;
        a.vel[i] = v;
      }
    }
  }
  if (!STATS) {  // vapour pairs are seen from both ends, wall pairs once: count 2 per pair
    const unsigned long long c = warp_sum((unsigned long long)(cvv + 2 * cvw));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.pair_count, c);
  }
}

// FP64, half list, packed: a warp owns 32 molecules (one lane each). Per window of kPackT list
// slots, an FP32 screen on the cell-local offsets drops the entries that are surely beyond the
// cutoff (FP32 r^2 at or above rc^2 (1 + 1e-5); the FP32 error is ~1e-7 of rc^2) and packs the
// others, molecule after molecule, into a per-warp queue; the FP64 pair terms then run over the
// queue with every lane busy, whatever the lanes' hit counts; finally each lane adds its own
// molecule's pair forces in list order (deterministic). Dropped vapour slots store a zero force
// for the partner's gather.
constexpr int kPackT = 8;
constexpr int kPackCap = 32 * kPackT;

struct PackWarp {
  dvec4 xi[32];                              // FP64 positions of the warp's molecules
  double rx[kPackCap], ry[kPackCap], rz[kPackCap];
  uint32_t qe[kPackCap];                     // list entry of each packed slot
  int32_t mi[32], mv[32], mr[32];            // molecule, vapour front length, replica
  uint16_t qmk[kPackCap];                    // (owner lane << 10) | list slot
};

__global__ void __launch_bounds__(256) k_forces_half_packed(Arrays a, PotDev p, int lpt) {
  extern __shared__ __align__(32) unsigned char pack_smem[];
  PackWarp& S = reinterpret_cast<PackWarp*>(pack_smem)[threadIdx.x >> 5];
  count_launch(a);
  clear_rebuild_flags(a);
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap, capv = p.cap_v;
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int chunk = next_chunk<32>(a); chunk >= 0; chunk = next_chunk<32>(a)) {
    const int t = chunk * 32 + lane;
    const bool live = t < N;
    int i = 0, n = 0, nvh = 0, r = 0;
    float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
      i = lpt ? MD_CHK(a, a.order[t], N) : t;
      n = a.n_front[i];
      nvh = a.n_vh[i];
      r = a.rep[i];
      li = a.lpos[i];
      S.xi[lane] = a.pos[i];
    }
    S.mi[lane] = i;
    S.mv[lane] = nvh;
    S.mr[lane] = r;
    const RepDev& R = a.reps[r];
    const float lcx = R.lcxf, lcy = R.lcyf, lcz = R.lczf;
    const int nmax = __reduce_max_sync(kFull, n);
    const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
    const uint32_t* __restrict__ fw = a.fwd + (size_t)i * capv;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    __syncwarp();
    for (int t0 = 0; t0 < nmax; t0 += kPackT) {
      // FP32 screen of the lane's own slots t0 .. t0 + kPackT - 1
      uint32_t e[kPackT];
      unsigned hm = 0;
#pragma unroll
      for (int s = 0; s < kPackT; ++s) {
        const int k = t0 + s;
        e[s] = 0u;
        if (k < n) {
          e[s] = row[k];
          const int j = MD_CHK(a, (int)(e[s] & kIndexMask), a.n_total + a.n_wall_total);
          const bool wall = j >= N;
          const float4 b = wall ? a.wlpos[j - N] : a.lpos[j];
          const float dx = (li.x - b.x) - cell_shift((e[s] >> 26) & 3u, lcx);
          const float dy = (li.y - b.y) - cell_shift((e[s] >> 28) & 3u, lcy);
          const float dz = (li.z - b.z) - cell_shift(e[s] >> 30, lcz);
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < (wall ? p.rcw2f_hi : p.rc2f_hi)) hm |= 1u << s;
          else if (k < nvh) a.pairbuf[MD_CHK(a, fw[k], (long long)a.n_total * p.cap_v + 1)] = make_dvec4(0.0, 0.0, 0.0, 0.0);
        }
      }
      // pack: the lane's survivors go to [seg, seg + c) of the queue, in slot order
      const int c = __popc(hm);
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int Q = __shfl_sync(kFull, incl, 31);
      const int seg = incl - c;
      int q = seg;
#pragma unroll
      for (int s = 0; s < kPackT; ++s) {
        if ((hm >> s) & 1u) {
          S.qe[q] = e[s];
          S.qmk[q] = (uint16_t)((lane << 10) | (t0 + s));
          ++q;
        }
      }
      __syncwarp();
      // FP64 pair terms over the queue: every lane takes a packed entry of any molecule
      for (int u = lane; u < Q; u += 32) {
        const uint32_t en = S.qe[u];
        const int mk = S.qmk[u];
        const int m = mk >> 10, k = mk & 1023;
        const dvec4 xm = S.xi[m];
        const RepDev& Rm = a.reps[S.mr[m]];
        const int j = MD_CHK(a, (int)(en & kIndexMask), a.n_total + a.n_wall_total);
        const bool wall = j >= N;
        const dvec4 xj = wall ? a.wpos[j - N] : a.pos[j];
        const double dx = image_hi(xm.x - xj.x, Rm.Lx, Rm.hi_thr_x);
        const double dy = image_hi(xm.y - xj.y, Rm.Ly, Rm.hi_thr_y);
        const double dz = xm.z - xj.z;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const bool in = lt_pos(r2, wall ? p.rcw2 : p.rc2);
        const double a12 = wall ? p.a12w : p.a12, b6 = wall ? p.b6w : p.b6;
        const double inv2 = rcp_nr(r2);
        const double inv6 = inv2 * inv2 * inv2;
        const double fr = in ? inv2 * inv6 * fma(a12, inv6, -b6) : 0.0;
        const double px = fr * dx, py = fr * dy, pz = fr * dz;
        S.rx[u] = px;
        S.ry[u] = py;
        S.rz[u] = pz;
        if (!wall && k < S.mv[m])
          a.pairbuf[MD_CHK(a, a.fwd[(size_t)S.mi[m] * capv + k], (long long)a.n_total * capv + 1)] = make_dvec4(px, py, pz, 0.0);
        cnt += in ? 1 : 0;
      }
      __syncwarp();
      // the lane's own molecule, in list order
      for (int u = seg; u < seg + c; ++u) {
        fx += S.rx[u];
        fy += S.ry[u];
        fz += S.rz[u];
      }
      __syncwarp();
    }
    if (live) a.fpart[i] = make_dvec4(fx, fy, fz, 0.0);
    __syncwarp();
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// FP64 observable pass over the full row (front + back): per-molecule energy and virial (half of
// each vapour pair to each end, wall pairs in full), pair counts and nearest wall atom. The forces
// of the last step are left untouched.
// With half rows (the atomic forms: no back region), each vapour pair is met once, at its lower
// end, which adds the partner's halves by atomics; the per-molecule sums start from zero.
template <int TPP>
__global__ void __launch_bounds__(256) k_stats_fp64(Arrays a, PotDev p, int half_rows) {
  count_launch(a);
  if (halted(a)) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = g / TPP, sub = g & (TPP - 1);
  const int N = a.n_total, cap = p.cap;
  const bool live = i < N;
  double pe = 0.0, vir = 0.0, pew = 0.0, virw = 0.0;
  double d2w = __longlong_as_double(0x7ff0000000000000ll);
  int cvv = 0, cvw = 0;
  if (live) {
    const RepDev& R = a.reps[a.rep[i]];
    const dvec4 xi = a.pos[i];
    const int nf = a.n_front[i], n = nf + a.n_back[i];
    const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
    for (int q = sub; q < n; q += TPP) {
      const int j = MD_CHK(a, (int)(row[q < nf ? q : cap - 1 - (q - nf)] & kIndexMask), a.n_total + a.n_wall_total);
      const bool wall = j >= N;
      const dvec4 xj = wall ? a.wpos[j - N] : a.pos[j];
      const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
      const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
      const double dz = xi.z - xj.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!lt_pos(r2, wall ? p.rcw2 : p.rc2)) continue;
      const double inv2 = 1.0 / r2, inv6 = inv2 * inv2 * inv2;
      if (wall) {
        const double fr = inv2 * inv6 * fma(p.a12w, inv6, -p.b6w);
        pew += inv6 * fma(p.e12w, inv6, -p.e6w) - p.ushift_w;
        virw += fr * r2;
        d2w = fmin(d2w, r2);
        ++cvw;
      } else {
        const double fr = inv2 * inv6 * fma(p.a12, inv6, -p.b6);
        const double hu = 0.5 * (inv6 * fma(p.e12, inv6, -p.e6) - p.ushift), hv = 0.5 * fr * r2;
        pe += hu;
        vir += hv;
        ++cvv;
        if (half_rows) {  // the partner's halves
          atomicAdd(&a.pe_i[j], hu);
          atomicAdd(&a.vir_i[j], hv);
          atomicAdd(&a.cnt_vv_i[j], 1);
        }
      }
    }
  }
  pe = group_sum<TPP>(pe);
  pew = group_sum<TPP>(pew);
  vir = group_sum<TPP>(vir);
  virw = group_sum<TPP>(virw);
  d2w = group_min<TPP>(d2w);
  cvv = group_sum<TPP>(cvv);
  cvw = group_sum<TPP>(cvw);
  if (!live || sub != 0) return;
  if (half_rows) {
    atomicAdd(&a.pe_i[i], pe);
    atomicAdd(&a.vir_i[i], vir);
    atomicAdd(&a.cnt_vv_i[i], cvv);
  } else {
    a.pe_i[i] = pe;
    a.vir_i[i] = vir;
    a.cnt_vv_i[i] = cvv;
  }
  a.pevw_i[i] = pew;
  a.virw_i[i] = virw;
  a.d2w_i[i] = d2w;
  a.cnt_vw_i[i] = cvw;
}

// f_i = (half-list sum) - (forces of the pairs held by lower partners, read contiguously from i's
// pairbuf row in i's back-region order); with
// KICK the second half-kick (Fig. 3) follows
template <bool KICK, int TPP>
__global__ void k_gather(Arrays a, PotDev p) {
  count_launch(a);
  if (KICK && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 0;  // this step kicks itself
  if (halted(a)) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = g / TPP, sub = g & (TPP - 1);
  const int N = a.n_total;
  const bool live = i < N;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  if (live) {
    const int m = min(a.n_back[i], p.cap_v);
    const dvec4* __restrict__ pb = a.pairbuf + (size_t)i * p.cap_v;
#pragma unroll 4
    for (int q = sub; q < m; q += TPP) {
      const dvec4 b = pb[q];
      fx += b.x;
      fy += b.y;
      fz += b.z;
    }
  }
  fx = group_sum<TPP>(fx);
  fy = group_sum<TPP>(fy);
  fz = group_sum<TPP>(fz);
  if (!live || sub != 0) return;
  dvec4 f = a.fpart[i];
  f.x -= fx;
  f.y -= fy;
  f.z -= fz;
  f.w = 0.0;
  a.frc[i] = f;
  if (KICK) {
    const RepDev& R = a.reps[a.rep[i]];
    dvec4 v = a.vel[i];
    const double h = R.half_dt_m;
    v.x += h * f.x;
    v.y += h * f.y;
    v.z += h * f.z;
    a.vel[i] = v;
  }
}

// Mixed precision, full list (front + back of the row): pair terms in FP32 from the cell-local FP32
// offsets (the displacement is (l_i - l_j) - dc * cell side, all terms small, so the rounding is
// relative to the cell size rather than the box), per-lane sums in compensated FP32 (TwoSum), the
// lanes of a molecule combined in FP64. Pairs whose FP32 r^2 lies within a relative 1e-5 of the
// cutoff are decided in FP64 from the FP64 positions, so the set of interacting pairs is the FP64
// one. The observable pass accumulates energies and virials in FP64 and measures wall distances in
// FP64.

template <bool STATS, bool KICK, int TPP>
__global__ void __launch_bounds__(256) k_forces_mixed(Arrays a, PotDev p, int lpt,
                                                      int half_rows) {
  constexpr int MPW = 32 / TPP;
  count_launch(a);
  clear_rebuild_flags(a);
  if (KICK && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 0;  // this step kicks itself
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap;
  const int lane = threadIdx.x & 31, sub = lane & (TPP - 1);
  int cnt = 0;
  for (int chunk = next_chunk<MPW>(a); chunk >= 0; chunk = next_chunk<MPW>(a)) {
    const int t = chunk * MPW + lane / TPP;
    const bool live = t < N;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    double pe = 0.0, vir = 0.0, pew = 0.0, virw = 0.0;
    double d2w = __longlong_as_double(0x7ff0000000000000ll);
    int cvv = 0, cvw = 0, i = 0;
    if (live) {
      i = lpt ? MD_CHK(a, a.order[t], N) : t;
      const RepDev& R = a.reps[a.rep[i]];
      const float4 li = a.lpos[i];
      const dvec4 xi = a.pos[i];
      const int nf = a.n_front[i], n = nf + a.n_back[i];
      const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      // software-pipelined as in the atomic form; slot q of the full row is the front's q-th
      // entry, then the back's from the end
      uint32_t e = sub < n ? row[sub < nf ? sub : cap - 1 - (sub - nf)] : 0u;
      float4 b = sub < n ? partner_lpos(a, e, N) : li;
      for (int q = sub; q < n; q += TPP) {
        const int qn = q + TPP;
        const uint32_t en = qn < n ? row[qn < nf ? qn : cap - 1 - (qn - nf)] : 0u;
        const float4 bn = qn < n ? partner_lpos(a, en, N) : li;
        const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
        const bool wall = j >= N;
        const float dx = (li.x - b.x) - cell_shift((e >> 26) & 3u, R.lcxf);
        const float dy = (li.y - b.y) - cell_shift((e >> 28) & 3u, R.lcyf);
        const float dz = (li.z - b.z) - cell_shift(e >> 30, R.lczf);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float lo = wall ? p.rcw2f_lo : p.rc2f_lo, hi = wall ? p.rcw2f_hi : p.rc2f_hi;
        bool in = r2 < lo;
        if (!in && r2 < hi) {
          const dvec4 xj = wall ? a.wpos[j - N] : a.pos[j];
          const double ex = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
          const double ey = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
          const double ez = xi.z - xj.z;
          in = ex * ex + ey * ey + ez * ez < (wall ? p.rcw2 : p.rc2);
        }
        if (in) {
          const float a12 = wall ? p.a12wf : p.a12f, b6 = wall ? p.b6wf : p.b6f;
          const float inv2 = __frcp_rn(r2);
          const float inv6 = inv2 * inv2 * inv2;
          const float fr = inv2 * inv6 * fmaf(a12, inv6, -b6);
          two_sum_acc(sx, cx, fr * dx);
          two_sum_acc(sy, cy, fr * dy);
          two_sum_acc(sz, cz, fr * dz);
          if (STATS) {
            const double u = (double)(inv6 * fmaf(wall ? p.e12wf : p.e12f, inv6,
                                                 -(wall ? p.e6wf : p.e6f)));
            if (wall) {
              const dvec4 xj = a.wpos[j - N];
              const double ex = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
              const double ey = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
              const double ez = xi.z - xj.z;
              pew += u - p.ushift_w;
              virw += (double)(fr * r2);
              d2w = fmin(d2w, ex * ex + ey * ey + ez * ez);
              ++cvw;
            } else {
              const double hu = 0.5 * (u - p.ushift), hv = 0.5 * (double)(fr * r2);
              pe += hu;
              vir += hv;
              ++cvv;
              if (half_rows) {  // half rows meet each vapour pair once: the partner's halves
                atomicAdd(&a.pe_i[j], hu);
                atomicAdd(&a.vir_i[j], hv);
                atomicAdd(&a.cnt_vv_i[j], 1);
              }
            }
          } else {
            cnt += wall ? 2 : 1;  // vapour pairs are seen from both ends
          }
        }
        e = en;
        b = bn;
      }
    }
    double fx = group_sum<TPP>(widen_f32(sx) + widen_f32(cx));
    double fy = group_sum<TPP>(widen_f32(sy) + widen_f32(cy));
    double fz = group_sum<TPP>(widen_f32(sz) + widen_f32(cz));
    if (STATS) {
      pe = group_sum<TPP>(pe);
      pew = group_sum<TPP>(pew);
      vir = group_sum<TPP>(vir);
      virw = group_sum<TPP>(virw);
      d2w = group_min<TPP>(d2w);
      cvv = group_sum<TPP>(cvv);
      cvw = group_sum<TPP>(cvw);
    }
    if (live && sub == 0) {
      if (!STATS) a.frc[i] = make_dvec4(fx, fy, fz, 0.0);  // the observable pass leaves forces
      if (KICK) {  // Fig. 3: v(t+dt) = v(t+dt/2) + a(t+dt) dt/2
        const RepDev& R = a.reps[a.rep[i]];
        dvec4 v = a.vel[i];
        const double h = R.half_dt_m;
        v.x += h * fx;
        v.y += h * fy;
        v.z += h * fz;
        a.vel[i] = v;
      }
      if (STATS) {
        if (half_rows) {
          atomicAdd(&a.pe_i[i], pe);
          atomicAdd(&a.vir_i[i], vir);
          atomicAdd(&a.cnt_vv_i[i], cvv);
        } else {
          a.pe_i[i] = pe;
          a.vir_i[i] = vir;
          a.cnt_vv_i[i] = cvv;
        }
        a.pevw_i[i] = pew;
        a.virw_i[i] = virw;
        a.d2w_i[i] = d2w;
        a.cnt_vw_i[i] = cvw;
      }
    }
  }
  if (!STATS) {
    const unsigned long long c = warp_sum((unsigned long long)cnt);
    if (lane == 0 && c) atomicAdd(a.pair_count, c);
  }
  finish_chunks(a);
}

// Mixed precision, half list, reaction forces by atomics: the pair terms of k_forces_mixed (FP32 on
// the cell-local offsets, the FP64 cutoff decision near rc) for the front of each row only -- every
// vapour pair once -- with the molecule's own sum in compensated FP32 and each pair's reaction
// (the FP32 pair force widened to FP64) sent to the partner by an FP64 atomic add. The forces must be
// zero beforehand; the summation order of the atomic adds varies from run to run.
template <int TPP>
__global__ void __launch_bounds__(256) k_forces_mixed_atomic(Arrays a, PotDev p, int lpt,
                                                             int owe_kick, int stat) {
  constexpr int MPW = 32 / TPP;
  count_launch(a);
  clear_rebuild_flags(a);
  if (owe_kick && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 1;
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap;
  const int lane = threadIdx.x & 31, sub = lane & (TPP - 1);
  int cnt = 0;
  ChunkWalk<MPW, TPP> walk;
  walk.start(a, stat, lpt);
  for (; walk.chunk >= 0; walk.advance(a, stat)) {
    const int chunk = walk.chunk;
    const int cnt0 = cnt;
    const int t = chunk * MPW + lane / TPP;
    const bool live = t < N;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int im = walk.take(a, stat, lpt, t);
    int i = 0;
    if (live) {
      i = im;
      const RepDev& R = a.reps[a.rep[i]];
      const float4 li = a.lpos[i];
      const dvec4 xi = a.pos[i];
      const int n = a.n_front[i], nvh = a.n_vh[i];
      const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      // software-pipelined: the next entry and its partner's offset load while this pair runs
      uint32_t e = sub < n ? row[sub] : 0u;
      float4 b = sub < n ? partner_lpos(a, e, N) : li;
      for (int q = sub; q < n; q += TPP) {
        const int qn = q + TPP;
        const uint32_t en = qn < n ? row[qn] : 0u;
        const float4 bn = qn < n ? partner_lpos(a, en, N) : li;
        const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
        const bool wall = j >= N;
        const float dx = (li.x - b.x) - cell_shift((e >> 26) & 3u, R.lcxf);
        const float dy = (li.y - b.y) - cell_shift((e >> 28) & 3u, R.lcyf);
        const float dz = (li.z - b.z) - cell_shift(e >> 30, R.lczf);
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float lo = wall ? p.rcw2f_lo : p.rc2f_lo, hi = wall ? p.rcw2f_hi : p.rc2f_hi;
        bool in = r2 < lo;
        if (!in && r2 < hi) {
          const dvec4 xj = wall ? a.wpos[j - N] : a.pos[j];
          const double ex = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
          const double ey = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
          const double ez = xi.z - xj.z;
          in = ex * ex + ey * ey + ez * ez < (wall ? p.rcw2 : p.rc2);
        }
        if (in) {
          const float a12 = wall ? p.a12wf : p.a12f, b6 = wall ? p.b6wf : p.b6f;
          const float inv2 = __frcp_rn(r2);
          const float inv6 = inv2 * inv2 * inv2;
          const float fr = inv2 * inv6 * fmaf(a12, inv6, -b6);
          const float px = fr * dx, py = fr * dy, pz = fr * dz;
          two_sum_acc(sx, cx, px);
          two_sum_acc(sy, cy, py);
          two_sum_acc(sz, cz, pz);
          if (q < nvh) {  // Newton's third law: the partner receives -p
            atomicAdd(&a.frc[j].x, widen_f32(-px));
            atomicAdd(&a.frc[j].y, widen_f32(-py));
            atomicAdd(&a.frc[j].z, widen_f32(-pz));
          }
          ++cnt;
        }
        e = en;
        b = bn;
      }
    }
    const double fx = group_sum<TPP>(widen_f32(sx) + widen_f32(cx));
    const double fy = group_sum<TPP>(widen_f32(sy) + widen_f32(cy));
    const double fz = group_sum<TPP>(widen_f32(sz) + widen_f32(cz));
    // a molecule with no pair within the cutoff adds nothing (dilute vapour: about half of them)
    const int found = group_sum<TPP>(cnt - cnt0);
    if (live && sub == 0 && found) {
      atomicAdd(&a.frc[i].x, fx);
      atomicAdd(&a.frc[i].y, fy);
      atomicAdd(&a.frc[i].z, fz);
    }
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// double-float remainder of list entry e's partner offset
__device__ __forceinline__ float4 partner_lpos_lo(const Arrays& a, uint32_t e, int N) {
  const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
  return j >= N ? a.wlpos_lo[j - N] : a.lpos_lo[j];
}

// the displacement (l_i - l_j) - shift as a double word, from the hi + lo parts of both offsets
// and of the cell shift: the hi differences by TwoSum (exact), the remainders added after
__device__ __forceinline__ dword dw_disp(float lih, float lil, float bh, float bl, float sh,
                                         float sl) {
  const dword t = two_sum(lih, -bh);
  const dword u = two_sum(t.hi, -sh);
  return two_sum(u.hi, ((t.lo + u.lo) + (lil - bl)) - sl);
}

// One double-float pair term (MD_PREC_DF64): whether list entry e (partner offsets b + bl) lies
// within the cutoff of molecule i (offsets li + ll) and, if so, the force on i as double words.
// The lanes screen with the FP32 offsets and decide the cutoff near rc in FP64, so the pair set is
// the FP64 one. Within the cutoff, the displacement (l_i - l_j) - dc*cell, r^2, 1/r^2, the LJ
// factor of Eq. 2 and the pair force run in double-word arithmetic on the hi + lo parts (~2^-44
// relative, against 2^-53 for FP64; the offsets themselves are exact to ~1e-14, like FP64
// positions in the box) -- work for the FP32 pipe, not the FP64 one.
__device__ __forceinline__ bool df_pair_term(const Arrays& a, const PotDev& p, const RepDev& R,
                                             int i, const float4& li, const float4& ll,
                                             uint32_t e, const float4& b, const float4& bl, int N,
                                             dword& px, dword& py, dword& pz) {
  const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
  const bool wall = j >= N;
  const uint32_t ox = (e >> 26) & 3u, oy = (e >> 28) & 3u, oz = e >> 30;
  const float shx = cell_shift(ox, R.lcxf), shy = cell_shift(oy, R.lcyf),
              shz = cell_shift(oz, R.lczf);
  const float dxf = (li.x - b.x) - shx, dyf = (li.y - b.y) - shy, dzf = (li.z - b.z) - shz;
  const float r2f = dxf * dxf + dyf * dyf + dzf * dzf;
  const float lo = wall ? p.rcw2f_lo : p.rc2f_lo, hi = wall ? p.rcw2f_hi : p.rc2f_hi;
  bool in = r2f < lo;
  if (!in && r2f < hi) {  // near rc: the FP64 decision, as the FP64 kernels take it
    const dvec4 xi = a.pos[i];
    const dvec4 xj = wall ? a.wpos[j - N] : a.pos[j];
    const double ex = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
    const double ey = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
    const double ez = xi.z - xj.z;
    in = lt_pos(ex * ex + ey * ey + ez * ez, wall ? p.rcw2 : p.rc2);
  }
  if (!in) return false;
  const dword dx = dw_disp(li.x, ll.x, b.x, bl.x, shx, cell_shift(ox, R.lcx_lo));
  const dword dy = dw_disp(li.y, ll.y, b.y, bl.y, shy, cell_shift(oy, R.lcy_lo));
  const dword dz = dw_disp(li.z, ll.z, b.z, bl.z, shz, cell_shift(oz, R.lcz_lo));
  const dword r2 = dw_add(dw_add(dw_sqr(dx), dw_sqr(dy)), dw_sqr(dz));
  const dword inv2 = dw_rcp(r2);
  const dword inv4 = dw_sqr(inv2);
  const dword inv6 = dw_mul(inv4, inv2);
  const dword inv8 = dw_sqr(inv4);
  const dword A = wall ? dword{p.a12wf, p.a12wl} : dword{p.a12f, p.a12l};
  const dword B = wall ? dword{-p.b6wf, -p.b6wl} : dword{-p.b6f, -p.b6l};
  const dword fr = dw_mul(inv8, dw_add(dw_mul(A, inv6), B));
  px = dw_mul(fr, dx);
  py = dw_mul(fr, dy);
  pz = dw_mul(fr, dz);
  return true;
}

// the molecule's own sum of double-word pair forces: a compensated FP32 pair per component
__device__ __forceinline__ void df_accumulate(float& s, float& c, const dword& p) {
  two_sum_acc(s, c, p.hi);
  c += p.lo;
}

// Double-float pair terms, half list, reaction forces by atomics: each vapour pair once, its
// reaction sent to the partner as an FP64 atomic add of the pair force's double-word value. The
// forces must be zero beforehand.
template <int TPP>
__global__ void __launch_bounds__(256) k_forces_df_atomic(Arrays a, PotDev p, int lpt,
                                                          int owe_kick, int stat) {
  constexpr int MPW = 32 / TPP;
  count_launch(a);
  clear_rebuild_flags(a);
  if (owe_kick && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 1;
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap;
  const int lane = threadIdx.x & 31, sub = lane & (TPP - 1);
  int cnt = 0;
  ChunkWalk<MPW, TPP> walk;
  walk.start(a, stat, lpt);
  for (; walk.chunk >= 0; walk.advance(a, stat)) {
    const int chunk = walk.chunk;
    const int cnt0 = cnt;
    const int t = chunk * MPW + lane / TPP;
    const bool live = t < N;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int im = walk.take(a, stat, lpt, t);
    int i = 0;
    if (live) {
      i = im;
      const RepDev& R = a.reps[a.rep[i]];
      const float4 li = a.lpos[i], ll = a.lpos_lo[i];
      const int n = a.n_front[i];
      const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      // software-pipelined: the next entry and its partner's offsets load while this pair runs
      uint32_t e = sub < n ? row[sub] : 0u;
      float4 b = sub < n ? partner_lpos(a, e, N) : li;
      float4 bl = sub < n ? partner_lpos_lo(a, e, N) : ll;
      for (int q = sub; q < n; q += TPP) {
        const int qn = q + TPP;
        const uint32_t en = qn < n ? row[qn] : 0u;
        const float4 bn = qn < n ? partner_lpos(a, en, N) : li;
        const float4 bln = qn < n ? partner_lpos_lo(a, en, N) : ll;
        dword px, py, pz;
        if (df_pair_term(a, p, R, i, li, ll, e, b, bl, N, px, py, pz)) {
          df_accumulate(sx, cx, px);
          df_accumulate(sy, cy, py);
          df_accumulate(sz, cz, pz);
          const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
          if (j < N) {  // Newton's third law: the partner receives -p
            atomicAdd(&a.frc[j].x, neg_bits(dw_to_double(px)));
            atomicAdd(&a.frc[j].y, neg_bits(dw_to_double(py)));
            atomicAdd(&a.frc[j].z, neg_bits(dw_to_double(pz)));
          }
          ++cnt;
        }
        e = en;
        b = bn;
        bl = bln;
      }
    }
    const double fx = group_sum<TPP>(widen_f32(sx) + widen_f32(cx));
    const double fy = group_sum<TPP>(widen_f32(sy) + widen_f32(cy));
    const double fz = group_sum<TPP>(widen_f32(sz) + widen_f32(cz));
    // a molecule with no pair within the cutoff adds nothing (dilute vapour: about half of them)
    const int found = group_sum<TPP>(cnt - cnt0);
    if (live && sub == 0 && found) {
      atomicAdd(&a.frc[i].x, fx);
      atomicAdd(&a.frc[i].y, fy);
      atomicAdd(&a.frc[i].z, fz);
    }
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// ------------------------------------------------------------------------------------------------
// The flat stream (force_tpp 64; atomic form), for dilute systems: a row there holds a few entries,
// and a kernel that walks molecules spends its time on each molecule's chain of dependent loads
// (its row's place, the row, the partners) with too few molecules per SM to hide it, and on lanes
// idling through other lanes' pair terms. Here the front rows of all molecules are copied at each
// rebuild into one stream -- entry k of it is list entry flat_ent[k] of molecule flat_own[k], the
// molecules in their stored (cell) order -- and the pair kernel splits the stream evenly: warp w of
// W takes tiles [w T / W, (w + 1) T / W) of the T tiles of 32 entries, so every warp has the same
// number of entries whatever the rows' lengths, with no work counter and no per-molecule loop. A
// lane loads its entries' owners and partners (kStreamBatch tiles at once), screens each entry in
// FP32 on the cell-local offsets and -- FP64 and double-float -- the entries that may lie within the
// cutoff (FP32 r^2 below rc^2 (1 + 1e-5)) join the warp's queue, a ring in shared memory; the pair
// terms run 32 at a time with every lane busy (the cutoff decided in FP64, Eq. 2 in FP64 or
// double-float words), FP64 with the positions of each round of 32 loaded while the round before
// it runs. The mixed form evaluates its FP32 pair terms where it screens them. Both ends of a pair receive its force by FP64 atomic adds (the owner
// +p, a vapour partner -p): no per-molecule sum, so no FP64 adds besides the pair term's own. The
// forces must be zero beforehand; the order of the adds varies from run to run.
constexpr int kStreamBatch = 4;   // tiles of 32 entries a lane loads before screening them

// The stream's fill, first pass: the front entries of each block of kFlatBlock molecules
__global__ void __launch_bounds__(kFlatBlock) k_flat_count(Arrays a, PotDev p) {
  count_launch(a);
  __shared__ int ws[kFlatBlock / 32];
  __shared__ int s_go;
  if (threadIdx.x == 0) s_go = !halted(a) && need_rebuild(a, p);
  __syncthreads();
  if (!s_go) return;  // (uniform in the block)
  const int i = blockIdx.x * kFlatBlock + threadIdx.x;
  int n = i < a.n_total ? a.n_front[i] : 0;
  n = warp_sum(n);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int t = warp_sum(ws[threadIdx.x]);
    if (threadIdx.x == 0) a.flat_part[blockIdx.x] = t;
  }
}

// Second pass: each block's place in the stream (the sum of the blocks before it), each molecule's
// place in its block (a block scan), then every warp copies its 32 rows, 32 entries at a time. The
// last block writes the stream's length.
__global__ void __launch_bounds__(kFlatBlock) k_flat_fill(Arrays a, PotDev p) {
  count_launch(a);
  __shared__ int ws[kFlatBlock / 32];
  __shared__ int s_base, s_go;
  if (threadIdx.x == 0) s_go = !halted(a) && need_rebuild(a, p);
  __syncthreads();
  if (!s_go) return;  // (uniform in the block)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // the sum of the earlier blocks' counts, in a fixed order
  int b = 0;
  for (int k = threadIdx.x; k < blockIdx.x; k += kFlatBlock) b += a.flat_part[k];
  b = warp_sum(b);
  if (lane == 0) ws[wid] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int t = warp_sum(ws[threadIdx.x]);
    if (threadIdx.x == 0) s_base = t;
  }
  __syncthreads();
  const int i = blockIdx.x * kFlatBlock + threadIdx.x;
  const int n = i < a.n_total ? a.n_front[i] : 0;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) ws[wid] = incl;  // (read below after the barrier; overwrites the sums above)
  __syncthreads();
  int wbase = s_base;
  for (int k = 0; k < wid; ++k) wbase += ws[k];
  const int excl = incl - n, T = __shfl_sync(kFull, incl, 31);
  const int cap = p.cap;
  for (int k0 = 0; k0 < T; k0 += 32) {
    const int k = k0 + lane;
    // the owner of warp entry k: the last lane whose prefix is at most k (its row is not empty)
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const int mid = (lo + hi + 1) >> 1;
      if (k >= __shfl_sync(kFull, excl, mid)) lo = mid;
      else hi = mid - 1;
    }
    const int slot = k - __shfl_sync(kFull, excl, lo);
    const int io = __shfl_sync(kFull, i, lo);
    const long long d = (long long)wbase + k;
    if (k < T && d >= a.flat_cap) atomicOr(a.status, kStatusOverflow);  // the stream is full
    if (k < T && d < a.flat_cap) {
      a.flat_ent[d] = a.nbr[(size_t)MD_CHK(a, io, a.n_total) * cap + MD_CHK(a, slot, cap)];
      a.flat_own[d] = io;
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kFlatBlock - 1)
    *a.n_flat = (int)min((long long)wbase + T, a.flat_cap);
}

// One FP64 pair term without a branch on the cutoff (the queued pairs of the flat stream: nearly
// all lie within it): the force on the owner, zero beyond the cutoff (decided in FP64); returns
// whether the pair lies within it.
__device__ __forceinline__ bool pair_term_nb(const PotDev& p, const RepDev& R, const dvec4& xi,
                                             const dvec4& xj, bool wall, unsigned act, double& px,
                                             double& py, double& pz) {
  double dx = xi.x - xj.x, dy = xi.y - xj.y;
  const double dz = xi.z - xj.z;
  // the periodic image's adds run only in a round where some lane's pair crosses an x or y edge
  // (rare in a stream in cell order); act: the lanes running this call
  const bool cross = ((uint32_t)__double2hiint(dx) & 0x7fffffffu) >= R.hi_thr_x ||
                     ((uint32_t)__double2hiint(dy) & 0x7fffffffu) >= R.hi_thr_y;
  if (__any_sync(act, cross)) {
    dx = image_hi(dx, R.Lx, R.hi_thr_x);
    dy = image_hi(dy, R.Ly, R.hi_thr_y);
  }
  const double r2 = dx * dx + dy * dy + dz * dz;
  const bool in = lt_pos(r2, wall ? p.rcw2 : p.rc2);
  const double a12 = wall ? p.a12w : p.a12, b6 = wall ? p.b6w : p.b6;
  const double inv2 = rcp_nr(r2);
  const double inv6 = inv2 * inv2 * inv2;
  const double fr = in ? inv2 * inv6 * fma(a12, inv6, -b6) : 0.0;
  px = fr * dx;
  py = fr * dy;
  pz = fr * dz;
  return in;
}

// One round of the FP64 flat stream's queue, held by a lane: the owner, its partner and their
// FP64 positions, loaded one round before the pair terms run
struct FlatRound {
  dvec4 xi, xj;
  int qi, j, rep;
};

template <int PREC>
__global__ void __launch_bounds__(256) k_forces_flat(Arrays a, PotDev p, int owe_kick) {
  // the warp's queue of screened pairs (FP64 and double-float): a ring in shared memory -- owner,
  // its replica, the list entry -- of which the Q from `head` on are waiting. FP64 keeps 128
  // slots: a round's positions load while the round before it runs (up to 63 wait, one round
  // loaded among them, before a push of 32)
  constexpr int kRing = PREC == kPrecFP64 ? 128 : 64;
  __shared__ int s_own[8][kRing], s_rep[8][kRing];
  __shared__ uint32_t s_ent[8][kRing];
  count_launch(a);
  clear_rebuild_flags(a);
  if (owe_kick && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 1;
  const int E = *a.n_flat;  // (loaded beside the status word: one round trip for both)
  if (halted(a)) return;
  const int N = a.n_total, lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long W = (long long)gridDim.x * (blockDim.x >> 5);
  const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  const long long tiles = (E + 31) >> 5;
  const int t0 = (int)(tiles * w / W), t1 = (int)(tiles * (w + 1) / W);
  int cnt = 0, Q = 0, head = 0;
  // FP64: the positions of the `n` slots from h, one per lane, into r (their loads in flight)
  auto load_round = [&](FlatRound& r, int h, int n) {
    if (lane < n) {
      const int slot = (h + lane) & (kRing - 1);
      r.qi = s_own[wib][slot];
      r.rep = s_rep[wib][slot];
      r.j = MD_CHK(a, (int)(s_ent[wib][slot] & kIndexMask), a.n_total + a.n_wall_total);
      r.xi = a.pos[r.qi];
      r.xj = r.j >= N ? a.wpos[r.j - N] : a.pos[r.j];
    }
  };
  // FP64: the pair terms of a loaded round of n slots, both ends' atomic adds
  auto run_round = [&](const FlatRound& r, int n) {
    const unsigned act = __ballot_sync(kFull, lane < n);
    if (lane < n) {
      double fx, fy, fz;
      if (pair_term_nb(p, a.reps[r.rep], r.xi, r.xj, r.j >= N, act, fx, fy, fz)) {
        atomicAdd(&a.frc[r.qi].x, fx);
        atomicAdd(&a.frc[r.qi].y, fy);
        atomicAdd(&a.frc[r.qi].z, fz);
        if (r.j < N) {  // Newton's third law: the partner receives -p
          atomicAdd(&a.frc[r.j].x, neg_bits(fx));
          atomicAdd(&a.frc[r.j].y, neg_bits(fy));
          atomicAdd(&a.frc[r.j].z, neg_bits(fz));
        }
        ++cnt;
      }
    }
  };
  // FP64: two round buffers used in turn (no register copies between them, so a round's loads
  // stay in flight while the other round runs); `ld` rounds (0 or 1) are loaded, from head on
  FlatRound rb[2];
  int ld = 0, cur = 0;
  // the pair terms of the next `n` waiting slots, one per lane (n <= 32): double-float
  auto evaluate = [&](int n) {
    __syncwarp();
    if (lane < n) {
      const int slot = (head + lane) & (kRing - 1);
      const int qi = s_own[wib][slot];
      const uint32_t qe = s_ent[wib][slot];
      const RepDev& RQ = a.reps[s_rep[wib][slot]];
      const int j = MD_CHK(a, (int)(qe & kIndexMask), a.n_total + a.n_wall_total);
      const float4 li = a.lpos[qi], ll = a.lpos_lo[qi];
      const float4 b = partner_lpos(a, qe, N), bl = partner_lpos_lo(a, qe, N);
      dword px, py, pz;
      const bool in = df_pair_term(a, p, RQ, qi, li, ll, qe, b, bl, N, px, py, pz);
      const double fx = dw_to_double(px), fy = dw_to_double(py), fz = dw_to_double(pz);
      if (in) {
        atomicAdd(&a.frc[qi].x, fx);
        atomicAdd(&a.frc[qi].y, fy);
        atomicAdd(&a.frc[qi].z, fz);
        if (j < N) {  // Newton's third law: the partner receives -p
          atomicAdd(&a.frc[j].x, neg_bits(fx));
          atomicAdd(&a.frc[j].y, neg_bits(fy));
          atomicAdd(&a.frc[j].z, neg_bits(fz));
        }
        ++cnt;
      }
    }
    head = (head + n) & (kRing - 1);
    Q -= n;
    __syncwarp();
  };
  // the lanes whose entry passed the screen (hit) append it to the ring in lane order. Double-float:
  // 32 waiting slots run (at most 31 wait before a push of at most 32). FP64: the first 32 are
  // loaded; once 64 wait, the next 32 load and the loaded round runs (at most 63 wait before a
  // push: 95 of 128 slots)
  auto push = [&](bool hit, int hi, int hr, uint32_t he) {
    const unsigned hm = __ballot_sync(kFull, hit);
    if (hit) {
      const int slot = (head + Q + __popc(hm & ((1u << lane) - 1u))) & (kRing - 1);
      s_own[wib][slot] = hi;
      s_rep[wib][slot] = hr;
      s_ent[wib][slot] = he;
    }
    Q += __popc(hm);
    if constexpr (PREC == kPrecFP64) {
      __syncwarp();
      if (!ld && Q >= 32) {  // (the first load: nothing ran yet, cur is 0)
        load_round(rb[0], head, 32);
        ld = 1;
      }
      if (ld && Q >= 64) {
        if (cur == 0) {
          load_round(rb[1], head + 32, 32);
          run_round(rb[0], 32);
        } else {
          load_round(rb[0], head + 32, 32);
          run_round(rb[1], 32);
        }
        cur ^= 1;
        head = (head + 32) & (kRing - 1);
        Q -= 32;
      }
      __syncwarp();
    } else {
      if (Q >= 32) evaluate(32);
    }
  };
  // a batch of kStreamBatch tiles: the entries and owners (the next batch's load while this one is
  // screened), then the owners' and partners' offsets
  uint32_t en[kStreamBatch];
  int on[kStreamBatch];
  auto load_batch = [&](int tb) {
#pragma unroll
    for (int u = 0; u < kStreamBatch; ++u) {
      const int k = (tb + u) * 32 + lane;
      const bool valid = tb + u < t1 && k < E;
      en[u] = valid ? a.flat_ent[k] : 0u;
      on[u] = valid ? MD_CHK(a, a.flat_own[k], N) : -1;
    }
  };
  if (t0 < t1) load_batch(t0);
  for (int tb = t0; tb < t1; tb += kStreamBatch) {
    uint32_t e[kStreamBatch];
    int own[kStreamBatch];
    float4 li[kStreamBatch], b[kStreamBatch];
    int rr[kStreamBatch];
#pragma unroll
    for (int u = 0; u < kStreamBatch; ++u) {
      e[u] = en[u];
      own[u] = on[u];
      const int i = own[u] >= 0 ? own[u] : 0;
      li[u] = a.lpos[i];
      rr[u] = a.rep[i];
      b[u] = partner_lpos(a, e[u], N);
    }
    if (tb + kStreamBatch < t1) load_batch(tb + kStreamBatch);  // (warp-uniform)
#pragma unroll
    for (int u = 0; u < kStreamBatch; ++u) {
      const RepDev& R = a.reps[rr[u]];
      const uint32_t eu = e[u];
      const int j = MD_CHK(a, (int)(eu & kIndexMask), a.n_total + a.n_wall_total);
      const bool wall = j >= N;
      const float dx = (li[u].x - b[u].x) - cell_shift((eu >> 26) & 3u, R.lcxf);
      const float dy = (li[u].y - b[u].y) - cell_shift((eu >> 28) & 3u, R.lcyf);
      const float dz = (li[u].z - b[u].z) - cell_shift(eu >> 30, R.lczf);
      const float r2 = dx * dx + dy * dy + dz * dz;
      const bool valid = own[u] >= 0;
      if constexpr (PREC == kPrecMixed) {
        const float lo = wall ? p.rcw2f_lo : p.rc2f_lo, hi = wall ? p.rcw2f_hi : p.rc2f_hi;
        bool in = valid && r2 < lo;
        if (valid && !in && r2 < hi) {  // near rc: the FP64 decision, as the FP64 kernels take it
          const dvec4 xi = a.pos[own[u]];
          const dvec4 xj = wall ? a.wpos[j - N] : a.pos[j];
          const double ex = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
          const double ey = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
          const double ez = xi.z - xj.z;
          in = lt_pos(ex * ex + ey * ey + ez * ez, wall ? p.rcw2 : p.rc2);
        }
        if (in) {
          const float a12 = wall ? p.a12wf : p.a12f, b6 = wall ? p.b6wf : p.b6f;
          const float inv2 = __frcp_rn(r2);
          const float inv6 = inv2 * inv2 * inv2;
          const float fr = inv2 * inv6 * fmaf(a12, inv6, -b6);
          const float px = fr * dx, py = fr * dy, pz = fr * dz;
          atomicAdd(&a.frc[own[u]].x, widen_f32(px));
          atomicAdd(&a.frc[own[u]].y, widen_f32(py));
          atomicAdd(&a.frc[own[u]].z, widen_f32(pz));
          if (!wall) {  // Newton's third law: the partner receives -p
            atomicAdd(&a.frc[j].x, widen_f32(-px));
            atomicAdd(&a.frc[j].y, widen_f32(-py));
            atomicAdd(&a.frc[j].z, widen_f32(-pz));
          }
          ++cnt;
        }
      } else {
        push(valid && r2 < (wall ? p.rcw2f_hi : p.rc2f_hi), own[u], rr[u], eu);
      }
    }
  }
  if constexpr (PREC == kPrecFP64) {
    // what is left: a loaded round and up to 31 more, or fewer than 32 unloaded
    __syncwarp();
    if (ld) {
      const int rest = Q - 32;  // in [0, 32)
      if (cur == 0) {
        load_round(rb[1], head + 32, rest);
        run_round(rb[0], 32);
        run_round(rb[1], rest);
      } else {
        load_round(rb[0], head + 32, rest);
        run_round(rb[1], 32);
        run_round(rb[0], rest);
      }
    } else if (Q) {
      load_round(rb[0], head, Q);
      run_round(rb[0], Q);
    }
  } else if constexpr (PREC != kPrecMixed) {
    if (Q) evaluate(Q);
  }
  const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
}

// Double-float pair terms, full list (front + back of each row), deterministic: every vapour
// pair is evaluated from both ends, with no atomics; each molecule sums its own row in slot order
// and writes its force, with the second half-kick fused when KICK (Fig. 3). The same sum from the
// same lists every run: bit-for-bit reproducible.
template <bool KICK, int TPP>
__global__ void __launch_bounds__(256) k_forces_df(Arrays a, PotDev p, int lpt) {
  constexpr int MPW = 32 / TPP;
  count_launch(a);
  clear_rebuild_flags(a);
  if (KICK && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 0;  // this step kicks itself
  if (halted(a)) return;
  const int N = a.n_total, cap = p.cap;
  const int lane = threadIdx.x & 31, sub = lane & (TPP - 1);
  int cnt = 0;
  for (int chunk = next_chunk<MPW>(a); chunk >= 0; chunk = next_chunk<MPW>(a)) {
    const int t = chunk * MPW + lane / TPP;
    const bool live = t < N;
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    int i = 0;
    if (live) {
      i = lpt ? MD_CHK(a, a.order[t], N) : t;
      const RepDev& R = a.reps[a.rep[i]];
      const float4 li = a.lpos[i], ll = a.lpos_lo[i];
      const int nf = a.n_front[i], n = nf + a.n_back[i];
      const uint32_t* __restrict__ row = a.nbr + (size_t)i * cap;
      // slot q of the full row is the front's q-th entry, then the back's from the end
      uint32_t e = sub < n ? row[sub < nf ? sub : cap - 1 - (sub - nf)] : 0u;
      float4 b = sub < n ? partner_lpos(a, e, N) : li;
      float4 bl = sub < n ? partner_lpos_lo(a, e, N) : ll;
      for (int q = sub; q < n; q += TPP) {
        const int qn = q + TPP;
        const uint32_t en = qn < n ? row[qn < nf ? qn : cap - 1 - (qn - nf)] : 0u;
        const float4 bn = qn < n ? partner_lpos(a, en, N) : li;
        const float4 bln = qn < n ? partner_lpos_lo(a, en, N) : ll;
        dword px, py, pz;
        if (df_pair_term(a, p, R, i, li, ll, e, b, bl, N, px, py, pz)) {
          df_accumulate(sx, cx, px);
          df_accumulate(sy, cy, py);
          df_accumulate(sz, cz, pz);
          cnt += (int)(e & kIndexMask) >= N ? 2 : 1;  // vapour pairs are seen from both ends
        }
        e = en;
        b = bn;
        bl = bln;
      }
    }
    const double fx = group_sum<TPP>(widen_f32(sx) + widen_f32(cx));
    const double fy = group_sum<TPP>(widen_f32(sy) + widen_f32(cy));
    const double fz = group_sum<TPP>(widen_f32(sz) + widen_f32(cz));
    if (live && sub == 0) {
      a.frc[i] = make_dvec4(fx, fy, fz, 0.0);
      if (KICK) {  // Fig. 3: v(t+dt) = v(t+dt/2) + a(t+dt) dt/2
        const RepDev& R = a.reps[a.rep[i]];
        dvec4 v = a.vel[i];
        const double h = R.half_dt_m;
        v.x += h * fx;
        v.y += h * fy;
        v.z += h * fz;
        a.vel[i] = v;
      }
    }
  }
  const unsigned long long c = warp_sum((unsigned long long)cnt);
  if (lane == 0 && c) atomicAdd(a.pair_count, c);
  finish_chunks(a);
}

// ------------------------------------------------------------------------------------------------
// Cell-tiled pair forces (pair_method 3): no Verlet list. A warp takes one row of cells (fixed iy,
// iz of one replica) and walks its molecules in chunks of at most 32, one lane per molecule. For a
// chunk spanning cells ix_lo .. ix_hi, the FP32 cell-local offsets of the vapour in the nine
// neighbouring rows (dy, dz in {-1, 0, 1}), cells ix_lo - 1 .. ix_hi + 1 with the periodic wrap,
// are staged in shared memory by coalesced float4 loads, each tagged with its molecule index. Every
// lane then tests every staged candidate of its own 27 cells in FP32 -- the displacement
// (l_i - l_j) - dc * cell side, exact as in the list build -- keeping the partners j > i (Newton's
// third law: each vapour pair once) and every wall atom of the 27 cells (read from L2, where lanes of
// one cell read the same addresses). A candidate whose FP32 r^2 lies below rc^2 (1 + 1e-5) goes to a
// per-warp queue; when 32 are queued (or the chunk is done) every lane takes one queued pair and
// evaluates its pair term in the context's precision -- FP64 on the FP64 positions, FP32 on the
// offsets, or double-float -- with the cutoff decided in FP64 near rc as in the list kernels, so
// the pair set is the FP64 one. The pair force goes to both molecules by FP64 atomic adds (the
// forces start from zero), which the L2 executes: the FP64 pipe does only pair terms, with every
// lane busy. With STATS the queue runs the FP64 observable terms instead (energy, virial, pair
// counts, nearest wall atom), added to both ends by atomics. Cells are the list cells (side at
// least max(rc, rc_w) + skin), rebuilt when a molecule has moved skin/2: every pair within the
// cutoff lies in neighbouring cells.
constexpr int kCellCap = 384;      // staged candidates per warp (vapour and wall atoms)
constexpr int kCellSlots = 34;     // cells along x a chunk may span, plus the two neighbours

// One staged neighbour run: row (dy, dz) of the chunk's row, vapour (runs 0-8) or wall atoms (runs
// 9-17), cells ix_lo - 1 .. ix_hi + 1 as three pieces -- [left cell][ix_lo .. ix_hi][right cell],
// x wrapped -- of the sorted arrays, staged from `base` (len 0: not staged).
struct CellRun {
  int s0, e0, s1, e1, s2, base, len, qb;   // piece starts / ends, staging offset, length, row
};

struct CellWarp {
  float4 ent[kCellCap];            // staged FP32 offsets (cp.async)
  int gid[kCellCap];               // their molecule or wall-atom index
  int raw[18][kCellSlots];         // per run: the CSR start of cells ix_lo .. ix_hi + 1 (cp.async)
  CellRun run[18];
  double ox[32], oy[32], oz[32];   // FP64 positions of the chunk's molecules
  float4 ol[32], oll[32];          // their FP32 offsets and double-float remainders
  float4 qb[32];                   // queued partner offset
  uint32_t qj[32];                 // queued partner: index | cell-offset code (list-entry packing)
  int32_t qo[32];                  // queued owner lane
};

// asynchronous global -> shared copies (cp.async): issued without holding registers, waited for
// once per chunk
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ int next_row(const Arrays& a) {
  int c = 0;
  if ((threadIdx.x & 31) == 0) c = atomicAdd(a.work, 1);
  c = __shfl_sync(kFull, c, 0);
  return c < a.n_rows ? c : -1;
}

// cell id of row `rb` (first cell of the row) at x index ix, wrapped
__device__ __forceinline__ int row_cell_at(int rb, int ix, int ncx) {
  return rb + (ix < 0 ? ix + ncx : (ix >= ncx ? ix - ncx : ix));
}

// the queued pairs, one per lane (lanes >= Q idle); forces, or with STATS the observable terms,
// added to both molecules by atomics. Returns the pairs within the cutoff this lane found.
template <int PREC, bool STATS>
__device__ int cell_flush(const Arrays& a, const PotDev& p, const RepDev& R, CellWarp& S, int Q,
                          int m0, int N) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  int found = 0;
  if (lane < Q) {
    const int o = S.qo[lane];
    const uint32_t e = S.qj[lane];
    const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
    const bool wall = j >= N;
    const int i = m0 + o;
    if (STATS || PREC == kPrecFP64) {
      const dvec4 xi = make_dvec4(S.ox[o], S.oy[o], S.oz[o], 0.0);
      const dvec4 xj = partner_pos(a, e, N);
      const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
      const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
      const double dz = xi.z - xj.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (lt_pos(r2, wall ? p.rcw2 : p.rc2)) {
        found = 1;
        const double inv2 = STATS ? 1.0 / r2 : rcp_nr(r2);
        const double inv6 = inv2 * inv2 * inv2;
        const double a12 = wall ? p.a12w : p.a12, b6 = wall ? p.b6w : p.b6;
        const double fr = inv2 * inv6 * fma(a12, inv6, -b6);
        if (STATS) {
          if (wall) {
            atomicAdd(&a.pevw_i[i], inv6 * fma(p.e12w, inv6, -p.e6w) - p.ushift_w);
            atomicAdd(&a.virw_i[i], fr * r2);
            atomicAdd(&a.cnt_vw_i[i], 1);
            atomicMin(reinterpret_cast<long long*>(&a.d2w_i[i]), __double_as_longlong(r2));
          } else {
            const double hu = 0.5 * (inv6 * fma(p.e12, inv6, -p.e6) - p.ushift);
            const double hv = 0.5 * fr * r2;
            atomicAdd(&a.pe_i[i], hu);
            atomicAdd(&a.vir_i[i], hv);
            atomicAdd(&a.cnt_vv_i[i], 1);
            atomicAdd(&a.pe_i[j], hu);
            atomicAdd(&a.vir_i[j], hv);
            atomicAdd(&a.cnt_vv_i[j], 1);
          }
        } else {
          const double px = fr * dx, py = fr * dy, pz = fr * dz;
          atomicAdd(&a.frc[i].x, px);
          atomicAdd(&a.frc[i].y, py);
          atomicAdd(&a.frc[i].z, pz);
          if (!wall) {  // Newton's third law: the partner receives -p
            atomicAdd(&a.frc[j].x, neg_bits(px));
            atomicAdd(&a.frc[j].y, neg_bits(py));
            atomicAdd(&a.frc[j].z, neg_bits(pz));
          }
        }
      }
    } else if (PREC == kPrecMixed) {
      const float4 li = S.ol[o], b = S.qb[lane];
      const float dx = (li.x - b.x) - cell_shift((e >> 26) & 3u, R.lcxf);
      const float dy = (li.y - b.y) - cell_shift((e >> 28) & 3u, R.lcyf);
      const float dz = (li.z - b.z) - cell_shift(e >> 30, R.lczf);
      const float r2 = dx * dx + dy * dy + dz * dz;
      bool in = r2 < (wall ? p.rcw2f_lo : p.rc2f_lo);
      if (!in) {  // the queue holds only r^2 below the upper band: decide in FP64
        const dvec4 xj = partner_pos(a, e, N);
        const double ex = image_hi(S.ox[o] - xj.x, R.Lx, R.hi_thr_x);
        const double ey = image_hi(S.oy[o] - xj.y, R.Ly, R.hi_thr_y);
        const double ez = S.oz[o] - xj.z;
        in = ex * ex + ey * ey + ez * ez < (wall ? p.rcw2 : p.rc2);
      }
      if (in) {
        found = 1;
        const float a12 = wall ? p.a12wf : p.a12f, b6 = wall ? p.b6wf : p.b6f;
        const float inv2 = __frcp_rn(r2);
        const float inv6 = inv2 * inv2 * inv2;
        const float fr = inv2 * inv6 * fmaf(a12, inv6, -b6);
        const float px = fr * dx, py = fr * dy, pz = fr * dz;
        atomicAdd(&a.frc[i].x, widen_f32(px));
        atomicAdd(&a.frc[i].y, widen_f32(py));
        atomicAdd(&a.frc[i].z, widen_f32(pz));
        if (!wall) {
          atomicAdd(&a.frc[j].x, widen_f32(-px));
          atomicAdd(&a.frc[j].y, widen_f32(-py));
          atomicAdd(&a.frc[j].z, widen_f32(-pz));
        }
      }
    } else {  // kPrecDF64
      dword px, py, pz;
      if (df_pair_term(a, p, R, i, S.ol[o], S.oll[o], e, S.qb[lane], partner_lpos_lo(a, e, N), N,
                       px, py, pz)) {
        found = 1;
        const double fx = dw_to_double(px), fy = dw_to_double(py), fz = dw_to_double(pz);
        atomicAdd(&a.frc[i].x, fx);
        atomicAdd(&a.frc[i].y, fy);
        atomicAdd(&a.frc[i].z, fz);
        if (!wall) {
          atomicAdd(&a.frc[j].x, neg_bits(fx));
          atomicAdd(&a.frc[j].y, neg_bits(fy));
          atomicAdd(&a.frc[j].z, neg_bits(fz));
        }
      }
    }
  }
  __syncwarp();
  return found;
}

// append this lane's hit (if any) to the queue, flushing the queue first when it would overflow
template <int PREC, bool STATS>
__device__ __forceinline__ void cell_push(const Arrays& a, const PotDev& p, const RepDev& R,
                                         CellWarp& S, int& Q, int& cnt, bool hit, uint32_t e,
                                         const float4& b, int m0, int N) {
  const unsigned hm = __ballot_sync(kFull, hit);
  if (!hm) return;
  const int lane = threadIdx.x & 31;
  const int c = __popc(hm);
  if (Q + c > 32) {
    cnt += cell_flush<PREC, STATS>(a, p, R, S, Q, m0, N);
    Q = 0;
  }
  if (hit) {
    const int u = Q + __popc(hm & ((1u << lane) - 1u));
    S.qj[u] = e;
    S.qo[u] = lane;
    S.qb[u] = b;
  }
  Q += c;
}

template <int PREC, bool STATS>
__global__ void __launch_bounds__(256) k_forces_cells(Arrays a, PotDev p, int owe_kick) {
  extern __shared__ __align__(16) unsigned char cell_smem[];
  CellWarp& S = reinterpret_cast<CellWarp*>(cell_smem)[threadIdx.x >> 5];
  count_launch(a);
  if (!STATS) clear_rebuild_flags(a);
  if (!STATS && owe_kick && blockIdx.x == 0 && threadIdx.x == 0) *a.kick_pending = 1;
  if (__syncthreads_or(halted(a) ? 1 : 0)) {  // uniform in the block: every block reports in
    finish_chunks(a);
    return;
  }
  const int N = a.n_total;
  const int lane = threadIdx.x & 31;
  int cnt = 0;
  for (int row = next_row(a); row >= 0; row = next_row(a)) {
    const int rb = a.row_cell[row];
    const RepDev& R = a.reps[a.cell_rep[rb]];
    const int ncx = R.ncx, ncy = R.ncy;
    const int rl = (rb - R.cell_off) / ncx;
    const int iy = rl % ncy, iz = rl / ncy;
    const int m_begin = a.vstart[rb], m_end = a.vstart[rb + ncx];
    int n = 0;
    for (int m0 = m_begin; m0 < m_end; m0 += n) {
      __syncwarp();  // every lane is done with the previous chunk's staging and queue
      // the chunk: at most 32 molecules spanning at most kCellSlots - 2 cells, whose neighbour
      // runs fit the staging (vapour always; wall atoms when some molecule has any nearby)
      n = min(32, m_end - m0);
      const int ix_lo = a.home[m0] & 1023;
      int ixl = ix_lo, wn = 0;
      if (lane < n) {
        ixl = a.home[m0 + lane] & 1023;
        wn = a.wnear[rb + ixl];
      }
      n = __popc(__ballot_sync(kFull, lane < n && ixl - ix_lo + 3 <= kCellSlots));
      int ix_hi = 0, len = 0, longest = 0, s0 = 0, e0 = 0, s1 = 0, e1 = 0, s2 = 0, qb = 0;
      for (;;) {
        ix_hi = __shfl_sync(kFull, ixl, n - 1);
        const bool walls = __any_sync(kFull, lane < n && wn > 0);
        // lane q < 18: run q's pieces (a vapour run holding only lower indices is left out)
        len = 0;
        const int kind = lane >= 9, r = lane % 9;
        const int jz = iz + r / 3 - 1;
        if (lane < 18 && jz >= 0 && jz < R.ncz && (!kind || walls)) {
          const int jy = (iy + r % 3 - 1 + ncy) % ncy;
          qb = R.cell_off + (jz * ncy + jy) * ncx;
          const int* __restrict__ arr = kind ? a.wstart : a.vstart;
          const int cl = row_cell_at(qb, ix_lo - 1, ncx), cr = row_cell_at(qb, ix_hi + 1, ncx);
          s0 = arr[cl];
          e0 = arr[cl + 1];
          s1 = arr[qb + ix_lo];
          e1 = arr[qb + ix_hi + 1];
          s2 = arr[cr];
          const int e2 = arr[cr + 1];
          if (kind || max(e0, max(e1, e2)) > m0) len = (e0 - s0) + (e1 - s1) + (e2 - s2);
        }
        // fewer molecules while a single run would not fit the staging (wall-heavy rows): every
        // run is then staged and screened in at most a few windows
        longest = __reduce_max_sync(kFull, len);
        if (longest <= kCellCap || n == 1) break;
        n = (n + 1) / 2;
      }
      const int W = ix_hi - ix_lo + 1;
      int total = 0;
      {  // the runs form one stream: run q starts at `base` (an exclusive scan of the lengths)
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        total = __shfl_sync(kFull, incl, 31);
        if (lane < 18) S.run[lane] = CellRun{s0, e0, s1, e1, s2, incl - len, len, qb};
      }
      __syncwarp();
      // the cell bounds of every run, and the chunk's molecules (loads in flight with the copies)
      for (int q = 0; q < 18; ++q) {
        const CellRun rq = S.run[q];
        if (rq.len == 0) continue;
        const int* __restrict__ arr = q >= 9 ? a.wstart : a.vstart;
        for (int c = lane; c <= W; c += 32) cp_async4(&S.raw[q][c], arr + rq.qb + ix_lo + c);
      }
      const bool own = lane < n;
      const int i = m0 + lane;
      float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
      const int ki = ixl - ix_lo + 1;  // the molecule's slot (1 .. W)
      if (own) {
        const dvec4 xi = a.pos[i];
        S.ox[lane] = xi.x;
        S.oy[lane] = xi.y;
        S.oz[lane] = xi.z;
        li = a.lpos[i];
        S.ol[lane] = li;
        if (PREC == kPrecDF64 && !STATS) S.oll[lane] = a.lpos_lo[i];
      }
      int Q = 0;
      const float r2v = p.rc2f_hi, r2w = p.rcw2f_hi;
      // the stream in windows of kCellCap entries: stage (asynchronous copies, one wait), then
      // every lane screens the staged part of its own 27 cells -- vapour partners j > i, then wall
      // atoms
      for (int w0 = 0; w0 < total; w0 += kCellCap) {
        const int w1 = min(total, w0 + kCellCap);
        __syncwarp();  // the previous window is screened
        for (int q = 0; q < 18; ++q) {
          const CellRun rq = S.run[q];
          const int k0 = max(0, w0 - rq.base), k1 = min(rq.len, w1 - rq.base);
          if (k0 >= k1) continue;
          const float4* __restrict__ src = q >= 9 ? a.wlpos : a.lpos;
          const int l0 = rq.e0 - rq.s0, l1 = rq.e1 - rq.s1;
          for (int k = k0 + lane; k < k1; k += 32) {
            const int g = MD_CHK(a, k < l0 ? rq.s0 + k : (k < l0 + l1 ? rq.s1 + (k - l0)
                                                                    : rq.s2 + (k - l0 - l1)),
                               q >= 9 ? a.n_wall_total : a.n_total);
            cp_async16(&S.ent[rq.base + k - w0], src + g);
            S.gid[rq.base + k - w0] = g;
          }
        }
        cp_async_wait_all();
        __syncwarp();
        for (int q = 0; q < 18; ++q) {
          const CellRun rq = S.run[q];
          const int k0 = max(0, w0 - rq.base), k1 = min(rq.len, w1 - rq.base);
          if (k0 >= k1) continue;
          const bool wall_run = q >= 9;
          const uint32_t cy = (uint32_t)((q % 9) % 3), cz = (uint32_t)((q % 9) / 3);
          const float sy = cell_shift(cy, R.lcyf), sz = cell_shift(cz, R.lczf);
          const int l0 = rq.e0 - rq.s0;
          // run-relative start of slot c (0: the left cell, 1 .. W: ix_lo .. ix_hi, W + 1: the
          // right cell)
          auto slot = [&](int c) {
            return c == 0 ? 0 : (c <= W + 1 ? l0 + (S.raw[q][c - 1] - rq.s1) : rq.len);
          };
          const int b1 = own ? slot(ki) : 0, b2 = own ? slot(ki + 1) : 0;
          const int lo = own ? max(slot(ki - 1), k0) : 0, hi = own ? min(slot(ki + 2), k1) : 0;
          const int trips = __reduce_max_sync(kFull, max(hi - lo, 0));
          const int off = rq.base - w0;
          for (int t = 0; t < trips; ++t) {
            const int k = lo + t;
            const bool valid = k < hi;
            const int kk = valid ? k + off : 0;
            const float4 b = S.ent[kk];
            const int g = S.gid[kk];
            const uint32_t cx = k < b1 ? 0u : (k < b2 ? 1u : 2u);
            const float dx = (li.x - b.x) - cell_shift(cx, R.lcxf);
            const float dy = (li.y - b.y) - sy, dz = (li.z - b.z) - sz;
            const float r2 = dx * dx + dy * dy + dz * dz;
            const bool hit = valid && (wall_run ? r2 < r2w : (g > i && r2 < r2v));
            const uint32_t e = (uint32_t)(wall_run ? N + g : g) | (cx << 26) | (cy << 28) |
                               (cz << 30);
            cell_push<PREC, STATS>(a, p, R, S, Q, cnt, hit, e, b, m0, N);
          }
        }
      }
      if (Q) cnt += cell_flush<PREC, STATS>(a, p, R, S, Q, m0, N);
    }
  }
  if (!STATS) {
    const unsigned long long c = warp_sum((unsigned long long)(2 * cnt));
    if (lane == 0 && c) atomicAdd(a.pair_count, c);
  }
  finish_chunks(a);
}

// the per-molecule observables the cell-tiled stats pass adds to by atomics start from zero (and
// the nearest wall distance from infinity)
__global__ void k_stats_init(Arrays a) {
  count_launch(a);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  a.pe_i[i] = 0.0;
  a.vir_i[i] = 0.0;
  a.pevw_i[i] = 0.0;
  a.virw_i[i] = 0.0;
  a.d2w_i[i] = __longlong_as_double(0x7ff0000000000000ll);
  a.cnt_vv_i[i] = 0;
  a.cnt_vw_i[i] = 0;
}

// ------------------------------------------------------------------------------------------------
// Small systems (pair_method 4, FP64, at most kSmallMax molecules): whole MD steps in one
// cooperative launch, no lists and no sorting. Per step, separated by the bounded grid barrier:
//   the owed Berendsen scaling of the previous step (partial sums, lambda at the barrier) and each
//   molecule's half-kick, drift, reflections and wrap (advance_molecule), writing its absolute FP32
//   position;
//   a warp per molecule: every vapour molecule of its replica and the wall atoms of the 27 cells
//   around it screened in FP32 on absolute positions (the periodic image taken in FP32, a screening
//   band of 2e-4 of rc^2 above the cutoff), the candidates queued and evaluated in FP64 with every
//   lane busy (pair_term: the FP64 cutoff decision and Eq. 2), the warp's sum -- a fixed
//   butterfly, so runs are bit-for-bit reproducible -- written as the molecule's force, and the
//   second half-kick (Fig. 3) applied.
// Each vapour pair is evaluated from both ends (no atomics). The paper's systems (2,184 and 2,800
// molecules, Sec. 4 and Sec. 5) are this size: their steps are bound by launch and memory latency,
// which one launch for many steps removes.
__device__ __forceinline__ bool any_thermo_due(const Arrays& a, long long s) {
  for (int r = 0; r < a.n_reps; ++r)
    if (thermo_due(a.reps[r], s)) return true;
  return false;
}

constexpr int kSmallStage = 2816;  // FP32 positions a block stages at a time (45 KB)

// The forces on molecules base .. base + 7, one per warp, with the second half-kick when KICK. The
// vapour of the block's replica (that of molecule `base`) is staged in shared memory in windows
// (cp.async) and screened from there; a molecule of another replica (a block straddling two) reads
// its replica's positions from global memory. The wall atoms of the 27 cells around a molecule are
// one stream: lanes 0-26 fetch the cells' ranges at once, and the lanes then walk the stream.
template <bool KICK>
__device__ int small_forces(const Arrays& a, const PotDev& p, uint32_t* sq, float4* stage, int base,
                            float rcs2, float rcws2, const dvec4* __restrict__ P,
                            const float4* __restrict__ XF) {
  const int lane = threadIdx.x & 31, N = a.n_total;
  const int i = base + (threadIdx.x >> 5);
  const bool live = i < N;
  const RepDev& RB = a.reps[a.rep[base]];
  const int ri = live ? a.rep[i] : a.rep[base];
  const bool staged = live && &a.reps[ri] == &RB;
  const RepDev& R = a.reps[ri];
  const dvec4 xi = live ? P[i] : make_dvec4(0.0, 0.0, 0.0, 0.0);
  const float4 xf = live ? XF[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float Lx = R.Lx, Ly = R.Ly, hx = R.hx, hy = R.hy;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  int cnt = 0, Q = 0;
  auto flush = [&]() {
    __syncwarp();
    if (lane < Q) {
      const uint32_t e = sq[lane];
      double px, py, pz;
      const int j = MD_CHK(a, (int)(e & kIndexMask), a.n_total + a.n_wall_total);
      if (pair_term(a, p, R, xi, e, j >= N ? a.wpos[j - N] : P[j], N, px, py, pz)) {
        fx += px;
        fy += py;
        fz += pz;
        cnt += j >= N ? 2 : 1;  // vapour pairs are met from both ends
      }
    }
    __syncwarp();
    Q = 0;
  };
  auto push = [&](bool hit, uint32_t e) {
    const unsigned hm = __ballot_sync(kFull, hit);
    if (!hm) return;
    const int c = __popc(hm);
    if (Q + c > 32) flush();
    if (hit) sq[Q + __popc(hm & ((1u << lane) - 1u))] = e;
    Q += c;
  };
  auto screen = [&](const float4& b, float lim) {
    float dx = xf.x - b.x, dy = xf.y - b.y;
    dx = dx >= hx ? dx - Lx : (dx < -hx ? dx + Lx : dx);
    dy = dy >= hy ? dy - Ly : (dy < -hy ? dy + Ly : dy);
    const float dz = xf.z - b.z;
    return dx * dx + dy * dy + dz * dz < lim;
  };
  // vapour of the block's replica, window by window (the loop is the block's)
  for (int w0 = RB.vap_off; w0 < RB.vap_off + RB.n_vap; w0 += kSmallStage) {
    const int w1 = min(w0 + kSmallStage, RB.vap_off + RB.n_vap);
    __syncthreads();  // the previous window is screened
    for (int k = threadIdx.x; k < w1 - w0; k += blockDim.x) cp_async16(&stage[k], &XF[w0 + k]);
    cp_async_wait_all();
    __syncthreads();
    if (staged)
      for (int j0 = w0; j0 < w1; j0 += 32) {
        const int j = j0 + lane;
        const bool valid = j < w1 && j != i;
        push(valid && screen(stage[valid ? j - w0 : 0], rcs2), (uint32_t)j);
      }
  }
  if (live && !staged)  // a molecule of another replica than the block's
    for (int j0 = R.vap_off; j0 < R.vap_off + R.n_vap; j0 += 32) {
      const int j = j0 + lane;
      const bool valid = j < R.vap_off + R.n_vap && j != i;
      push(valid && screen(XF[valid ? j : i], rcs2), (uint32_t)j);
    }
  if (live && R.n_wall > 0) {  // the wall atoms of the 27 cells around the molecule
    const int ix = min(max((int)floorf((xf.x + hx) / R.lcxf), 0), R.ncx - 1);
    const int iy = min(max((int)floorf((xf.y + hy) / R.lcyf), 0), R.ncy - 1);
    const int iz = min(max((int)floorf((xf.z + (float)R.hz) / R.lczf), 0), R.ncz - 1);
    int ws = 0, nw = 0;
    if (lane < 27) {
      const int jz = iz + lane / 9 - 1;
      if (jz >= 0 && jz < R.ncz) {
        const int jy = (iy + (lane / 3) % 3 - 1 + R.ncy) % R.ncy;
        const int jx = (ix + lane % 3 - 1 + R.ncx) % R.ncx;
        const int cn = R.cell_off + (jz * R.ncy + jy) * R.ncx + jx;
        ws = a.wstart[cn];
        nw = a.wstart[cn + 1] - ws;
      }
    }
    int incl = nw;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - nw, T = __shfl_sync(kFull, incl, 31);
    constexpr int kBatch = 4;  // stream entries a lane loads before screening them
    for (int k0 = 0; k0 < T; k0 += 32 * kBatch) {
      int w[kBatch];
      float4 b[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int k = k0 + 32 * u + lane;
        // the cell holding stream entry k: the last cell whose stream start is at most k
        int lo = 0, hi = 26;
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int mid = (lo + hi + 1) >> 1;
          if (k >= __shfl_sync(kFull, excl, mid)) lo = mid;
          else hi = mid - 1;
        }
        // (every lane takes part in the shuffles; the result is kept only inside the stream)
        const int wk = __shfl_sync(kFull, ws, lo) + (k - __shfl_sync(kFull, excl, lo));
        w[u] = k < T ? wk : -1;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) b[u] = a.wxf[w[u] >= 0 ? w[u] : 0];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        push(w[u] >= 0 && screen(b[u], rcws2), (uint32_t)(N + (w[u] >= 0 ? w[u] : 0)));
    }
  }
  if (Q) flush();
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  fz = warp_sum(fz);
  if (live && lane == 0) {
    a.frc[i] = make_dvec4(fx, fy, fz, 0.0);
    if (KICK) {  // Fig. 3: v(t+dt) = v(t+dt/2) + a(t+dt) dt/2
      dvec4 v = a.vel[i];
      kick_v(v, make_dvec4(fx, fy, fz, 0.0), R.half_dt_m);
      a.vel[i] = v;
    }
  }
  return cnt;
}

__global__ void __launch_bounds__(256) k_small_steps(Arrays a, PotDev p, int nsteps) {
  __shared__ uint32_t sq[8][32];
  __shared__ __align__(16) float4 stage[kSmallStage];
  count_launch(a);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nb8 = gridDim.x * (blockDim.x >> 5);  // molecules the grid takes per round
  const float rcs2 = (float)(p.rc2 * (1.0 + 2e-4)), rcws2 = (float)(p.rcw2 * (1.0 + 2e-4));
  // the step counter, the owed kick and thermostat, read by every block before any block writes
  // (block 0 writes them back only at the end, after the first step's barrier, which every block
  // reaches having read them: no barrier is needed before the first step)
  const long long s0 = *reinterpret_cast<volatile long long*>(a.step);
  int pend = *reinterpret_cast<volatile const int32_t*>(a.kick_pending);
  long long owed = thermo_owed(a);
  bool ok = true;
  int cnt = 0;
  if (nsteps == 0) {  // the forces at the current positions (md_compute_forces): positions may
                      // have been loaded or re-sorted since the last step wrote their FP32 copy
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_total; i += gridDim.x * blockDim.x) {
      const dvec4 x = a.pos[i];
      a.xf[i] = make_float4(narrow_f64(x.x), narrow_f64(x.y), narrow_f64(x.z), 0.f);
    }
    ok = thermo_barrier(a, p, 0);
    const bool halt = __syncthreads_or(halted(a) ? 1 : 0) != 0;  // uniform in the block
    for (int base = blockIdx.x * 8; ok && !halt && base < a.n_total; base += nb8)
      cnt += small_forces<false>(a, p, sq[wib], stage, base, rcs2, rcws2, a.pos, a.xf);
  }
  // A block owns the molecules whose forces it takes (base + warp, base = its first 8, then every
  // nb8 on) and advances exactly those, so a molecule's kick and its next drift are the same
  // block's: one grid barrier a step (every position advanced before any force), with the
  // positions in two buffers -- step k reads one and writes the other -- so that a block advancing
  // into the new buffer never overwrites a position another block is still reading.
  for (int k = 0; k < nsteps && ok; ++k) {
    const long long s = s0 + k + 1;
    const dvec4* xin = (k & 1) ? a.pos_alt : a.pos;
    dvec4* xout = (k & 1) ? a.pos : a.pos_alt;
    float4* xfout = (k & 1) ? a.xf : a.xf_alt;
    if (owed) {  // the previous step's thermostat: v(t+dt)^2 per (replica, chunk), lambda
      if (k > 0) {  // every block's kick of the previous step is written
        ok = thermo_barrier(a, p, 0);
        if (!ok) break;
      }
      const int units = a.n_reps * a.rep_chunks;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int r = u / a.rep_chunks, ch = u % a.rep_chunks;
        const RepDev& R = a.reps[r];
        if (!thermo_due(R, owed) || ch * 1024 >= R.n_vap) continue;
        const double t = thermo_chunk_sum(a, R, ch * 1024, min(R.n_vap, ch * 1024 + 1024), pend);
        if (threadIdx.x == 0) a.rep_part[(size_t)u * 8] = t;
      }
      ok = thermo_barrier(a, p, owed);
      if (!ok) break;
    }
    const bool halt = __syncthreads_or(halted(a) ? 1 : 0) != 0;  // uniform in the block
    for (int r = threadIdx.x >> 3; !halt; r += blockDim.x >> 3) {
      const int i = (blockIdx.x + r * gridDim.x) * 8 + (threadIdx.x & 7);
      if (i >= a.n_total) break;
      advance_molecule(a, i, pend, owed, kIntAbsolute, xin, xout, xfout);
    }
    ok = thermo_barrier(a, p, 0);
    if (!ok) break;
    for (int base = blockIdx.x * 8; !halt && base < a.n_total; base += nb8)
      cnt += small_forces<true>(a, p, sq[wib], stage, base, rcs2, rcws2, xout, xfout);
    __syncthreads();  // this block's kicks are written before it advances its molecules again
    pend = 0;
    owed = any_thermo_due(a, s) ? s : 0;
  }
  // an odd number of steps left the positions in the second buffer: each block copies its own
  // (nothing reads the first buffer after the last step's barrier)
  if (nsteps & 1) {
    for (int r = threadIdx.x >> 3;; r += blockDim.x >> 3) {
      const int i = (blockIdx.x + r * gridDim.x) * 8 + (threadIdx.x & 7);
      if (i >= a.n_total) break;
      a.pos[i] = a.pos_alt[i];
      a.xf[i] = a.xf_alt[i];
    }
  }
  const unsigned long long c = warp_sum((unsigned long long)cnt);
  if (lane == 0 && c && nsteps > 0) atomicAdd(a.pair_count, c);
  if (blockIdx.x == 0 && threadIdx.x == 0 && nsteps > 0) {
    *a.step = s0 + nsteps;
    *a.kick_pending = 0;                      // every step kicked itself
    *a.thermo_owed = halted(a) ? 0 : owed;    // the last step's scaling, paid later
  }
}


// ------------------------------------------------------------------------------------------------
// observables: pore assignment, occupancy, adsorbed count, axial profile (integer atomics: exact)

__global__ void k_observe(Arrays a, PotDev p) {
  count_launch(a);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  const RepDev& R = a.reps[a.rep[i]];
  const dvec4 x = a.pos[i];
  int g = 0;
  double best = __longlong_as_double(0x7ff0000000000000ll);
  for (int q = 0; q < R.n_pores; ++q) {
    const PoreDev& P = a.pores[R.pore_off + q];
    const double dx = wrap_diff(x.x - P.cx, R.Lx, R.hx);
    const double dy = wrap_diff(x.y - P.cy, R.Ly, R.hy);
    const double d2 = P.kind == 3 ? dy * dy : dx * dx + dy * dy;
    if (d2 < best) {
      best = d2;
      g = q;
    }
    if (fabs(x.z) < R.slab_half && in_pore(P.kind, P.r0, P.r1, P.r_cavity, P.width, dx, dy, x.z,
                                           R.slab_half))
      atomicAdd(&a.occ[R.pore_off + q], 1ull);
  }
  if (a.d2w_i[i] < p.r_ads2) atomicAdd(&a.ads[R.group_off + g], 1ull);
  int b = (int)floor((x.z + R.hz) / R.bin_width);
  b = b < 0 ? 0 : (b >= R.n_bins ? R.n_bins - 1 : b);
  atomicAdd(&a.prof[(size_t)R.prof_off + (size_t)g * R.n_bins + b], 1ull);
}

// per-replica sums in a fixed order: blocks (replica, chunk of 1024 molecules) write partials,
// one block per replica adds them in chunk order. Quantities: ke, pe_vv, pe_vw, vir_vv, vir_vw,
// ordered vapour pair count, wall pair count.
__global__ void __launch_bounds__(256) k_rep_partial(Arrays a, PotDev p) {
  count_launch(a);
  const int r = blockIdx.x / a.rep_chunks, ch = blockIdx.x % a.rep_chunks;
  const RepDev& R = a.reps[r];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const int k0 = ch * 1024, k1 = min(R.n_vap, k0 + 1024);
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int i = R.vap_off + k;
    const dvec4 v = a.vel[i];
    acc[0] += v.x * v.x + v.y * v.y + v.z * v.z;
    acc[1] += a.pe_i[i];
    acc[2] += a.pevw_i[i];
    acc[3] += a.vir_i[i];
    acc[4] += a.virw_i[i];
    acc[5] += (double)a.cnt_vv_i[i];
    acc[6] += (double)a.cnt_vw_i[i];
  }
  __shared__ double sh[7][8];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const double w = warp_sum(acc[q]);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
    a.rep_part[(size_t)blockIdx.x * 8 + threadIdx.x] = t;
  }
}

__global__ void k_rep_final(Arrays a, PotDev p) {
  count_launch(a);
  const int r = blockIdx.x;
  if (threadIdx.x < 7) {
    double t = 0.0;
    for (int ch = 0; ch < a.rep_chunks; ++ch)
      t += a.rep_part[((size_t)r * a.rep_chunks + ch) * 8 + threadIdx.x];
    a.rep_sums[r * 8 + threadIdx.x] = threadIdx.x == 0 ? 0.5 * p.mass * t : t;
  }
}

// virial pressure per pore (Sec. 2): P_q = (sum m v^2 + sum W_i) / (d V_q) over the molecules
// inside pore q (the occupancy predicate), W_i = vir_i + virw_i. Blocks (replica, chunk) write
// partial sums for every pore of the replica, one thread per pore adds them in chunk order.
__global__ void __launch_bounds__(256) k_pore_partial(Arrays a, PotDev p) {
  count_launch(a);
  const int r = blockIdx.x / a.rep_chunks, ch = blockIdx.x % a.rep_chunks;
  const RepDev& R = a.reps[r];
  if (R.n_pores == 0) return;
  __shared__ double sh[8];
  const int k0 = ch * 1024, k1 = min(R.n_vap, k0 + 1024);
  for (int q = 0; q < R.n_pores; ++q) {
    const PoreDev& P = a.pores[R.pore_off + q];
    double acc = 0.0;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      const int i = R.vap_off + k;
      const dvec4 x = a.pos[i];
      if (!(fabs(x.z) < R.slab_half)) continue;
      const double dx = wrap_diff(x.x - P.cx, R.Lx, R.hx);
      const double dy = wrap_diff(x.y - P.cy, R.Ly, R.hy);
      if (!in_pore(P.kind, P.r0, P.r1, P.r_cavity, P.width, dx, dy, x.z, R.slab_half)) continue;
      const dvec4 v = a.vel[i];
      acc += p.mass * (v.x * v.x + v.y * v.y + v.z * v.z) + a.vir_i[i] + a.virw_i[i];
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
      a.pore_part[(size_t)blockIdx.x * a.max_pores + q] = t;
    }
    __syncthreads();
  }
}

__global__ void k_pore_final(Arrays a) {
  count_launch(a);
  const int r = blockIdx.x;
  const RepDev& R = a.reps[r];
  for (int q = threadIdx.x; q < R.n_pores; q += blockDim.x) {
    double t = 0.0;
    for (int ch = 0; ch < a.rep_chunks; ++ch)
      t += a.pore_part[((size_t)r * a.rep_chunks + ch) * a.max_pores + q];
    const double vol = a.pores[R.pore_off + q].vol;
    a.pore_press[R.pore_off + q] = vol > 0.0 ? t / ((double)R.dims * vol) : 0.0;
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers

void launch_small_steps(const Arrays& a, const PotDev& p, const Tuning& t, int nsteps,
                        cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::max(1, std::min(nblocks(a.n_total, 8),
                                                    t.sm_count * t.small_blocks_per_sm)));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_small_steps, a, p, nsteps);
}

// the step kernel's grid: every block resident at once (its thermostat barrier waits for all of
// them), at most what covers the molecules once
int integrate_grid(const Arrays& a, const Tuning& t) {
  return std::max(1, std::min(nblocks(a.n_total, 256), t.sm_count * t.integrate_blocks_per_sm));
}

// launched as a cooperative kernel: the runtime refuses a grid whose blocks cannot all be resident
// at once (the barrier's bounded wait is the second line of defence)
void launch_barrier_check(const Arrays& a, const PotDev& p, cudaStream_t s) {
  k_barrier_check<<<2, 32, 0, s>>>(a, p);
}

void launch_integrate_first(const Arrays& a, const PotDev& p, bool mixed, const StepConds& c,
                            int flags, const Tuning& t, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)integrate_grid(a, t));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (mixed)
    cudaLaunchKernelEx(&cfg, k_integrate_first<true>, a, p, c, flags);
  else
    cudaLaunchKernelEx(&cfg, k_integrate_first<false>, a, p, c, flags);
}

bool flat_form(bool mixed, const Tuning& t);

void launch_rebuild(const Arrays& a, const PotDev& p, const Tuning& t, bool mixed, cudaStream_t s) {
  const int b = 256;
  const int nt = nblocks(a.n_total, b);
  const int ntiles = nblocks(a.n_cells, 4096);
  // the pair kernel walks the front of each row (FP64, or mixed with atomic reaction forces) or the
  // whole row (mixed, deterministic): the processing order sorts by that length
  // (double-float pair terms in the deterministic form walk the whole row, as mixed does)
  const int half = ((!mixed && !t.df64) || t.atomic_acc) ? 1 : 0, lpt = t.lpt;
  k_cell_clear<<<nt, b, 0, s>>>(a, p);
  k_cell_count<<<nt, b, 0, s>>>(a, p);
  if (ntiles <= 16) {
    k_scan_single<<<1, 1024, 0, s>>>(a, p);
  } else {
    k_scan_tiles<<<ntiles, 1024, 0, s>>>(a, p);
    k_scan_top<<<1, 1024, 0, s>>>(a, p, ntiles);
    k_scan_add<<<ntiles, 1024, 0, s>>>(a, p);
  }
  k_scatter<<<nt, b, 0, s>>>(a, p);
  k_permute<<<nt, b, 0, s>>>(a, p, t.cells);
  if (t.cells) return;  // the cell method walks the sorted cells themselves: no lists, no order
  // the atomic forms walk only the front of each row: half rows
  // the flat stream needs no processing order; its fill runs for it (and for the tuner's timings)
  const bool flat = flat_form(mixed, t);
  const int order = lpt && (!flat || t.flat_fill) ? 1 : 0;
  // the two list builds: the device runs the one that suits the occupancy (or the tuning's)
  k_list_build<<<std::min(nblocks(a.n_cells, kListWarps), t.sm_count * 16), kListWarps * 32, 0, s>>>(
      a, p, half, t.atomic_acc, order, t.list_mode);
  k_list_build_mol<<<nblocks(a.n_total, kListThreads), kListThreads, 0, s>>>(
      a, p, half, t.atomic_acc, order, t.list_mode);
  if (order) k_order_assign<<<nt, b, 0, s>>>(a, p, half);
  if (!mixed && !t.df64 && !t.atomic_acc) k_fwd_build<<<std::min(nblocks(a.n_total, 8), t.sm_count * 8), 256, 0, s>>>(a, p);
  if (a.flat_ent && (flat || t.flat_fill)) {  // the front rows as one stream
    const int nf = std::max(1, nblocks(a.n_total, kFlatBlock));
    k_flat_count<<<nf, kFlatBlock, 0, s>>>(a, p);
    k_flat_fill<<<nf, kFlatBlock, 0, s>>>(a, p);
  }
}

// the per-molecule pair observables that half rows accumulate by atomics start from zero
void zero_pair_stats(const Arrays& a, cudaStream_t s) {
  cudaMemsetAsync(a.pe_i, 0, sizeof(double) * (size_t)a.n_total, s);
  cudaMemsetAsync(a.vir_i, 0, sizeof(double) * (size_t)a.n_total, s);
  cudaMemsetAsync(a.cnt_vv_i, 0, sizeof(int32_t) * (size_t)a.n_total, s);
}

// grid of the pair kernels: at most SMs x blocks per SM; warps fetch chunks of molecules
int pair_grid(long long threads, int block, int per_sm, const Tuning& t) {
  return std::min(nblocks(threads, block), std::max(1, t.sm_count * per_sm));
}

template <int TPP>
void launch_mixed(const Arrays& a, const PotDev& p, bool stats, bool kick, const Tuning& t,
                  cudaStream_t s) {
  const int b = t.force_block;
  const int g = pair_grid((long long)a.n_total * TPP, b, t.force_blocks_per_sm_mixed, t);
  if (!stats && t.atomic_acc) {
    // forces start from zero (k_integrate_first clears them in a step); the second half-kick of
    // a step is deferred into the next first half-kick
    if (!kick) k_zero_forces<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
    k_forces_mixed_atomic<TPP><<<g, b, 0, s>>>(a, p, t.lpt, kick ? 1 : 0, t.static_chunks);
    return;
  }
  if (stats) {
    if (t.atomic_acc) zero_pair_stats(a, s);
    k_forces_mixed<true, false, TPP><<<g, b, 0, s>>>(a, p, t.lpt, t.atomic_acc);
  } else if (kick) {
    k_forces_mixed<false, true, TPP><<<g, b, 0, s>>>(a, p, t.lpt, 0);
  } else {
    k_forces_mixed<false, false, TPP><<<g, b, 0, s>>>(a, p, t.lpt, 0);
  }
}

// FP64: half-list pass (TPP lanes per molecule, or the packed kernel for TPP = 32), then the
// gather (with the second half-kick when KICK)
template <int TPP>
void launch_fp64(const Arrays& a, const PotDev& p, bool kick, const Tuning& t, cudaStream_t s) {
  const int b = t.force_block;
  const int per_sm = t.force_blocks_per_sm_fp64;
  if (t.atomic_acc) {
    // forces start from zero: k_integrate_first clears them on the way through a step
    if (!kick) k_zero_forces<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
    // in a step the second half-kick is deferred into the next first half-kick
    if constexpr (TPP == 32) {
      const size_t sm = (size_t)(b / 32) * sizeof(AtomicQueue);
      k_forces_atomic_packed<<<pair_grid((long long)a.n_total * kAqLanes, b, per_sm, t), b, sm,
                               s>>>(a, p, t.lpt, kick ? 1 : 0);
    } else {
      k_forces_half_atomic<TPP><<<pair_grid((long long)a.n_total * TPP, b, per_sm, t), b, 0,
                                  s>>>(a, p, t.lpt, kick ? 1 : 0, t.static_chunks);
    }
    return;
  }
  if constexpr (TPP == 32) {
    const size_t sm = (size_t)(b / 32) * sizeof(PackWarp);
    k_forces_half_packed<<<pair_grid(a.n_total, b, per_sm, t), b, sm, s>>>(a, p, t.lpt);
  } else {
    k_forces_half<TPP><<<pair_grid((long long)a.n_total * TPP, b, per_sm, t), b, 0, s>>>(a, p,
                                                                                       t.lpt);
  }
  const int gb = nblocks((long long)a.n_total * t.gather_tpp, 256);
  switch (t.gather_tpp) {
    case 1:
      if (kick) k_gather<true, 1><<<gb, 256, 0, s>>>(a, p);
      else k_gather<false, 1><<<gb, 256, 0, s>>>(a, p);
      break;
    case 2:
      if (kick) k_gather<true, 2><<<gb, 256, 0, s>>>(a, p);
      else k_gather<false, 2><<<gb, 256, 0, s>>>(a, p);
      break;
    default:
      if (kick) k_gather<true, 4><<<gb, 256, 0, s>>>(a, p);
      else k_gather<false, 4><<<gb, 256, 0, s>>>(a, p);
      break;
  }
}

// FP64 context with double-float pair terms: atomic reaction forces, or the full-list form
template <int TPP>
void launch_df(const Arrays& a, const PotDev& p, bool kick, const Tuning& t, cudaStream_t s) {
  const int b = t.force_block;
  const int g = pair_grid((long long)a.n_total * TPP, b, t.force_blocks_per_sm_fp64, t);
  if (!t.atomic_acc) {
    if (kick) k_forces_df<true, TPP><<<g, b, 0, s>>>(a, p, t.lpt);
    else k_forces_df<false, TPP><<<g, b, 0, s>>>(a, p, t.lpt);
    return;
  }
  // forces start from zero (k_integrate_first clears them in a step); the second half-kick of a
  // step is deferred into the next first half-kick
  if (!kick) k_zero_forces<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
  k_forces_df_atomic<TPP><<<g, b, 0, s>>>(a, p, t.lpt, kick ? 1 : 0, t.static_chunks);
}

// the cell-tiled kernels: one warp's shared memory is a CellWarp
size_t cell_smem(int block) { return (size_t)(block / 32) * sizeof(CellWarp); }

int cell_prec(bool mixed, const Tuning& t) {
  return mixed ? kPrecMixed : (t.df64 ? kPrecDF64 : kPrecFP64);
}

int cell_grid(const Arrays& a, bool mixed, const Tuning& t) {
  const int per_sm = mixed ? t.force_blocks_per_sm_mixed : t.force_blocks_per_sm_fp64;
  return pair_grid((long long)std::max(a.n_rows, 1) * 32, t.force_block, per_sm, t);
}

template <bool STATS>
void launch_cells_kernel(const Arrays& a, const PotDev& p, bool mixed, const Tuning& t, int owe,
                         cudaStream_t s) {
  const int b = t.force_block, g = cell_grid(a, mixed, t);
  const size_t sm = cell_smem(b);
  switch (cell_prec(mixed, t)) {
    case kPrecMixed: k_forces_cells<kPrecMixed, STATS><<<g, b, sm, s>>>(a, p, owe); break;
    case kPrecDF64: k_forces_cells<kPrecDF64, STATS><<<g, b, sm, s>>>(a, p, owe); break;
    default: k_forces_cells<kPrecFP64, STATS><<<g, b, sm, s>>>(a, p, owe); break;
  }
}

void launch_cells(const Arrays& a, const PotDev& p, bool mixed, bool stats, bool kick,
                  const Tuning& t, cudaStream_t s) {
  if (stats) {
    k_stats_init<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
    launch_cells_kernel<true>(a, p, mixed, t, 0, s);
    return;
  }
  // forces start from zero (k_integrate_first clears them in a step); the second half-kick of a
  // step is deferred into the next first half-kick
  if (!kick) k_zero_forces<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
  launch_cells_kernel<false>(a, p, mixed, t, kick ? 1 : 0, s);
}

// the flat stream (force_tpp 64, atomic form): the front rows as one stream, split evenly
bool flat_form(bool mixed, const Tuning& t) {
  return t.atomic_acc && !t.cells && !t.small && !t.all_pairs &&
         (mixed ? t.tpp_mixed : t.tpp_fp64) == kFlatTpp;
}

void launch_flat(const Arrays& a, const PotDev& p, bool mixed, int owe, const Tuning& t,
                 cudaStream_t s) {
  // the warps split the stream evenly: SMs x blocks per SM blocks, whatever the stream's length
  const int b = t.force_block;
  const int g = std::max(1, t.sm_count * (mixed ? t.force_blocks_per_sm_mixed
                                                : t.force_blocks_per_sm_fp64));
  if (mixed) k_forces_flat<kPrecMixed><<<g, b, 0, s>>>(a, p, owe);
  else if (t.df64) k_forces_flat<kPrecDF64><<<g, b, 0, s>>>(a, p, owe);
  else k_forces_flat<kPrecFP64><<<g, b, 0, s>>>(a, p, owe);
}

void launch_forces(const Arrays& a, const PotDev& p, bool mixed, bool stats, bool kick,
                   const Tuning& t, cudaStream_t s) {
  if (!stats && flat_form(mixed, t)) {
    // forces start from zero (k_integrate_first clears them in a step); the second half-kick of
    // a step is deferred into the next first half-kick
    if (!kick) k_zero_forces<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
    launch_flat(a, p, mixed, kick ? 1 : 0, t, s);
    return;
  }
  if (t.small) {  // (a step kicks inside the small-system kernel: here the forces alone)
    if (stats) k_allpairs<true, false><<<nblocks(a.n_total, 128), 128, 0, s>>>(a, p);
    else launch_small_steps(a, p, t, 0, s);
    return;
  }
  if (t.cells) {
    launch_cells(a, p, mixed, stats, kick, t, s);
    return;
  }
  if (mixed) {
    switch (t.tpp_mixed) {
      case 1: launch_mixed<1>(a, p, stats, kick, t, s); break;
      case 2: launch_mixed<2>(a, p, stats, kick, t, s); break;
      case 8: launch_mixed<8>(a, p, stats, kick, t, s); break;
      case 16: launch_mixed<16>(a, p, stats, kick, t, s); break;
      default: launch_mixed<4>(a, p, stats, kick, t, s); break;
    }
    return;
  }
  if (t.all_pairs) {
    const int g = nblocks(a.n_total, 128);
    if (stats) k_allpairs<true, false><<<g, 128, 0, s>>>(a, p);
    else if (kick) k_allpairs<false, true><<<g, 128, 0, s>>>(a, p);
    else k_allpairs<false, false><<<g, 128, 0, s>>>(a, p);
    return;
  }
  if (stats) {  // FP64 observables: a full-row pass that leaves the forces untouched
    if (t.atomic_acc) zero_pair_stats(a, s);
    k_stats_fp64<4><<<nblocks((long long)a.n_total * 4, 256), 256, 0, s>>>(a, p, t.atomic_acc);
    return;
  }
  if (t.df64) {
    switch (t.tpp_fp64) {
      case 1: launch_df<1>(a, p, kick, t, s); break;
      case 2: launch_df<2>(a, p, kick, t, s); break;
      case 8: launch_df<8>(a, p, kick, t, s); break;
      case 16: launch_df<16>(a, p, kick, t, s); break;
      default: launch_df<4>(a, p, kick, t, s); break;
    }
    return;
  }
  switch (t.tpp_fp64) {
    case 1: launch_fp64<1>(a, p, kick, t, s); break;
    case 2: launch_fp64<2>(a, p, kick, t, s); break;
    case 8: launch_fp64<8>(a, p, kick, t, s); break;
    case 16: launch_fp64<16>(a, p, kick, t, s); break;
    case 32: launch_fp64<32>(a, p, kick, t, s); break;
    default: launch_fp64<4>(a, p, kick, t, s); break;
  }
}

template <int TPP>
void pair_pass_tpp(const Arrays& a, const PotDev& p, bool mixed, const Tuning& t, cudaStream_t s) {
  const int b = t.force_block;
  if (mixed) {
    const int gm = pair_grid((long long)a.n_total * TPP, b, t.force_blocks_per_sm_mixed, t);
    if (t.atomic_acc) k_forces_mixed_atomic<TPP><<<gm, b, 0, s>>>(a, p, t.lpt, 0, t.static_chunks);
    else k_forces_mixed<false, false, TPP><<<gm, b, 0, s>>>(a, p, t.lpt, 0);
    return;
  }
  const int g = pair_grid((long long)a.n_total * TPP, b, t.force_blocks_per_sm_fp64, t);
  if (t.df64 && t.atomic_acc) k_forces_df_atomic<TPP><<<g, b, 0, s>>>(a, p, t.lpt, 0, t.static_chunks);
  else if (t.df64) k_forces_df<false, TPP><<<g, b, 0, s>>>(a, p, t.lpt);
  else if (t.atomic_acc) k_forces_half_atomic<TPP><<<g, b, 0, s>>>(a, p, t.lpt, 0, t.static_chunks);
  else k_forces_half<TPP><<<g, b, 0, s>>>(a, p, t.lpt);
}

void launch_pair_pass(const Arrays& a, const PotDev& p, bool mixed, const Tuning& t,
                      cudaStream_t s) {
  if (flat_form(mixed, t)) {
    launch_flat(a, p, mixed, 0, t, s);
    return;
  }
  if (t.small) {
    launch_small_steps(a, p, t, 0, s);
    return;
  }
  if (t.cells) {
    launch_cells_kernel<false>(a, p, mixed, t, 0, s);
    return;
  }
  if (!mixed && t.all_pairs) {
    k_allpairs<false, false><<<nblocks(a.n_total, 128), 128, 0, s>>>(a, p);
    return;
  }
  const int tpp = mixed ? t.tpp_mixed : t.tpp_fp64;
  if (!mixed && tpp == 32) {
    const int g = pair_grid((long long)a.n_total * (t.atomic_acc ? kAqLanes : 1), t.force_block,
                            t.force_blocks_per_sm_fp64, t);
    if (t.atomic_acc) {
      const size_t sm = (size_t)(t.force_block / 32) * sizeof(AtomicQueue);
      k_forces_atomic_packed<<<g, t.force_block, sm, s>>>(a, p, t.lpt, 0);
    } else {
      const size_t sm = (size_t)(t.force_block / 32) * sizeof(PackWarp);
      k_forces_half_packed<<<g, t.force_block, sm, s>>>(a, p, t.lpt);
    }
    return;
  }
  switch (tpp) {
    case 1: pair_pass_tpp<1>(a, p, mixed, t, s); break;
    case 2: pair_pass_tpp<2>(a, p, mixed, t, s); break;
    case 8: pair_pass_tpp<8>(a, p, mixed, t, s); break;
    case 16: pair_pass_tpp<16>(a, p, mixed, t, s); break;
    default: pair_pass_tpp<4>(a, p, mixed, t, s); break;
  }
}

// ------------------------------------------------------------------------------------------------
// state transfer: caller-order xyz arrays <-> cell-sorted device records

// caller rows [off, off + n) staged for a state load, checked before they replace anything: every
// position inside its replica's box (x and y in [-L/2, L/2), z in [-Lz/2, Lz/2]; NaN fails), for a
// planar replica y = vy = 0, and every velocity component finite. The lowest offending row lands
// in *bad as 3 k (outside the box), 3 k + 1 (off the plane) or 3 k + 2 (a non-finite velocity);
// *bad keeps kNoBadRow when every row passes.
__global__ void k_check_state(Arrays a, const double* __restrict__ xin,
                              const double* __restrict__ vin, int off, int n, int* bad) {
  count_launch(a);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = off + k;
  const RepDev& R = a.reps[a.rep[i]];
  const double x = xin[3 * (size_t)i], y = xin[3 * (size_t)i + 1], z = xin[3 * (size_t)i + 2];
  const double vx = vin[3 * (size_t)i], vy = vin[3 * (size_t)i + 1], vz = vin[3 * (size_t)i + 2];
  int code = -1;
  if (!(x >= -R.hx && x < R.hx && y >= -R.hy && y < R.hy && z >= -R.hz && z <= R.hz))
    code = 3 * k;
  else if (R.dims == 2 && (y != 0.0 || vy != 0.0))
    code = 3 * k + 1;
  else if (!(isfinite(vx) && isfinite(vy) && isfinite(vz)))
    code = 3 * k + 2;
  if (code >= 0) atomicMin(bad, code);
}

// molecules [off, off + n) take the caller-order rows xin/vin (xyz interleaved, same offset); the
// stored order restarts as the caller's (id = index within the replica), forces cleared. Nothing
// is loaded when k_check_state found a bad row.
__global__ void k_load_state(Arrays a, const double* __restrict__ xin,
                             const double* __restrict__ vin, int off, int n, const int* bad) {
  count_launch(a);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || *bad != kNoBadRow) return;
  const int i = off + k;
  const dvec4 x = make_dvec4(xin[3 * (size_t)i], xin[3 * (size_t)i + 1], xin[3 * (size_t)i + 2],
                             0.0);
  a.pos[i] = x;
  // the skin check's reference, from the molecule's current home cell (a rebuild follows a load)
  a.lref[i] = local_offset(a, a.reps[a.rep[i]], x, a.home[i]);
  a.vel[i] = make_dvec4(vin[3 * (size_t)i], vin[3 * (size_t)i + 1], vin[3 * (size_t)i + 2], 0.0);
  a.frc[i] = make_dvec4(0.0, 0.0, 0.0, 0.0);
  a.id[i] = i - a.reps[a.rep[i]].vap_off;
  if (k == 0) *a.kick_pending = 0;  // owed kicks were settled before the load
}

// The load that keeps the stored order (the list methods): record i takes the caller row of the
// molecule it holds (row vap_off + id[i] of xin/vin), so the lists, cells and stream still name the
// right molecules; its FP32 offsets are refreshed and its displacement from its position at the
// last build is tested as a step tests it -- the replicas where some molecule lies at least skin/2
// away are flagged (those past the grouping threshold with them), and the chain that follows
// rebuilds only those, so the lists stay complete (every pair within rc is listed while no
// molecule is skin/2 from its reference). Forces cleared. Nothing is loaded when k_check_state
// found a bad row.
__global__ void k_load_state_keep(Arrays a, PotDev p, const double* __restrict__ xin,
                                  const double* __restrict__ vin, int off, int n, const int* bad) {
  count_launch(a);
  if (*bad != kNoBadRow) return;  // (the same word for every thread)
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int trig = 0;
  if (k < n) {
    const int i = off + k;
    const int r = a.rep[i];
    const RepDev& R = a.reps[r];
    const size_t row = MD_CHK(a, (size_t)R.vap_off + (size_t)a.id[i], (size_t)a.n_total);
    const dvec4 x = make_dvec4(xin[3 * row], xin[3 * row + 1], xin[3 * row + 2], 0.0);
    a.pos[i] = x;
    a.vel[i] = make_dvec4(vin[3 * row], vin[3 * row + 1], vin[3 * row + 2], 0.0);
    a.frc[i] = make_dvec4(0.0, 0.0, 0.0, 0.0);
    float4 lhi, llo;
    local_offset_df(a, R, x, a.home[i], lhi, llo);
    a.lpos[i] = lhi;
    a.lpos_lo[i] = llo;
    const float4 r0 = a.lref[i];
    const float dx = lhi.x - r0.x, dy = lhi.y - r0.y, dz = lhi.z - r0.z;
    const double d2 = widen_f32(dx * dx + dy * dy + dz * dz);
    if (ge_pos(d2, p.group_disp2))
      atomicMax(&a.rep_disp2[r], (unsigned long long)__double_as_longlong(d2));
    trig = ge_pos(d2, p.half_skin2) ? 1 : 0;
  }
  if (__syncthreads_or(trig) && threadIdx.x == 0) atomicExch(a.force_rebuild, 1);
  if (k == 0) *a.kick_pending = 0;  // owed kicks were settled before the load
}

// out rows (caller order, xyz interleaved) of molecules [off, off + n) from the records src
__global__ void k_store_rows(Arrays a, const dvec4* __restrict__ src, double* __restrict__ out,
                             int off, int n) {
  count_launch(a);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = off + k;
  const size_t row = MD_CHK(a, (size_t)a.reps[a.rep[i]].vap_off + (size_t)a.id[i], a.n_total);
  const dvec4 v = src[i];
  out[3 * row] = v.x;
  out[3 * row + 1] = v.y;
  out[3 * row + 2] = v.z;
}

void launch_load_state(const Arrays& a, const PotDev& p, const double* xin, const double* vin,
                       int off, int n, int* bad, bool keep_order, cudaStream_t s) {
  if (n <= 0) return;
  k_check_state<<<nblocks(n, 256), 256, 0, s>>>(a, xin, vin, off, n, bad);
  if (keep_order)
    k_load_state_keep<<<nblocks(n, 256), 256, 0, s>>>(a, p, xin, vin, off, n, bad);
  else
    k_load_state<<<nblocks(n, 256), 256, 0, s>>>(a, xin, vin, off, n, bad);
}

void launch_store_rows(const Arrays& a, const dvec4* src, double* out, int off, int n,
                       cudaStream_t s) {
  if (n > 0) k_store_rows<<<nblocks(n, 256), 256, 0, s>>>(a, src, out, off, n);
}

// one-time kernel attributes (before any launch or capture); *integrate_per_sm receives how many
// blocks of the step kernel an SM holds at once
cudaError_t configure_kernels(int* integrate_per_sm, int* small_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(
      k_forces_half_packed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * sizeof(PackWarp)));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_forces_atomic_packed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(8 * sizeof(AtomicQueue)));
  if (e != cudaSuccess) return e;
  const int cs = (int)cell_smem(256);
  if ((e = cudaFuncSetAttribute(k_forces_cells<kPrecFP64, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_forces_cells<kPrecMixed, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_forces_cells<kPrecDF64, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_forces_cells<kPrecFP64, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_forces_cells<kPrecMixed, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_forces_cells<kPrecDF64, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) != cudaSuccess)
    return e;
  int o1 = 0, o2 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_integrate_first<false>, 256, 0);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_integrate_first<true>, 256, 0);
  if (e != cudaSuccess) return e;
  *integrate_per_sm = std::max(1, std::min(o1, o2));
  int o3 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o3, k_small_steps, 256, 0);
  if (e != cudaSuccess) return e;
  *small_per_sm = std::max(1, o3);
  return cudaSuccess;
}

void launch_settle(const Arrays& a, const PotDev& p, cudaStream_t s) {
  k_kick_pending<<<nblocks(a.n_total, 256), 256, 0, s>>>(a, p);  // the thermostat reads v(t+dt)
  k_thermo_partial<<<a.n_reps * a.rep_chunks, 256, 0, s>>>(a);
  k_thermo_lambda<<<nblocks(a.n_reps, 8), 256, 0, s>>>(a, p);
  k_thermo_scale<<<nblocks(a.n_total, 256), 256, 0, s>>>(a);
  cudaMemsetAsync(a.thermo_owed, 0, sizeof(long long), s);  // paid
}

void launch_observables(const Arrays& a, const PotDev& p, cudaStream_t s) {
  const int b = 256;
  k_observe<<<nblocks(a.n_total, b), b, 0, s>>>(a, p);
  k_rep_partial<<<a.n_reps * a.rep_chunks, 256, 0, s>>>(a, p);
  k_rep_final<<<a.n_reps, 32, 0, s>>>(a, p);
  k_pore_partial<<<a.n_reps * a.rep_chunks, 256, 0, s>>>(a, p);
  k_pore_final<<<a.n_reps, 32, 0, s>>>(a);
}

}  // namespace mdk
