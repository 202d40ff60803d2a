// md_kernels.cu -- CUDA kernels (sm_103a) of the pore / water-vapour MD step.
//
// One MD step (Sec. 2 velocity Verlet, Figs. 1-4 of arXiv:1812.07993), all replicas per launch:
//   k_integrate_first   half-kick + drift (Fig. 2), z reflection, x/y wrap, displacement max
//   rebuild chain       only when a molecule moved >= skin/2 since the last build (decided on
//                       the device; the kernels return at once otherwise):
//                         k_cell_count -> k_scan_* -> k_scatter -> k_permute -> k_copyback ->
//                         k_list_build (warp per cell)
//   k_forces_*          Lennard-Jones forces at r(t+dt) (Eq. 2, Fig. 1) from the Verlet lists
//   k_integrate_second  half-kick (Fig. 3)
//   k_thermo_reduce / k_thermo_scale   Berendsen scaling on thermostat steps (Fig. 4)
// None of these kernels spins or waits on another block.
#include <cstdint>
#include <cuda_runtime.h>

#include "md_internal.cuh"

namespace mdk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool halted(const Arrays& a) {
  return *reinterpret_cast<volatile const int32_t*>(a.status) != 0;
}

__device__ __forceinline__ bool need_rebuild(const Arrays& a, const PotDev& p) {
  if (*a.force_rebuild) return true;
  return __longlong_as_double((long long)*a.max_disp2) >= p.half_skin2;
}

// periodic image of a coordinate difference of two wrapped positions (|d| < L): the high word of
// |d| is compared against the high word of L/2 -- an integer test, no FP64 instruction. Pairs in a
// list are either closer than the list radius or further than L minus it, far from L/2.
__device__ __forceinline__ double image_hi(double d, double L, uint32_t thr) {
  const int hw = __double2hiint(d);
  if ((uint32_t)(hw & 0x7fffffff) >= thr) d += (hw < 0) ? L : -L;
  return d;
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

__device__ __forceinline__ void cell_center(const RepDev& R, int home, double& cx, double& cy,
                                            double& cz) {
  const int ix = home & 1023, iy = (home >> 10) & 1023, iz = (home >> 20) & 1023;
  cx = -R.hx + (ix + 0.5) * R.lcx;
  cy = -R.hy + (iy + 0.5) * R.lcy;
  cz = -R.hz + (iz + 0.5) * R.lcz;
}

__device__ __forceinline__ float4 local_offset(const RepDev& R, const dvec4& x, int home) {
  double cx, cy, cz;
  cell_center(R, home, cx, cy, cz);
  float4 l;
  l.x = (float)wrap_diff(x.x - cx, R.Lx, R.hx);
  l.y = (float)wrap_diff(x.y - cy, R.Ly, R.hy);
  l.z = (float)(x.z - cz);
  l.w = 0.f;
  return l;
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

// ------------------------------------------------------------------------------------------------
// Fig. 2: v(t+dt/2) = v + a dt/2 ; r(t+dt) = r + v(t+dt/2) dt  (the same r(t+dt) as r + v dt + a dt^2/2)
template <bool MIXED>
__global__ void k_integrate_first(Arrays a, PotDev p) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.step += 1;
    *a.any_scale = 0;
  }
  if (halted(a)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double d2 = 0.0;
  if (i < a.n_total) {
    const RepDev& R = a.reps[a.rep[i]];
    dvec4 x = a.pos[i], v = a.vel[i];
    const dvec4 f = a.frc[i];
    const double h = 0.5 * R.dt * p.inv_mass;
    v.x += h * f.x;
    v.y += h * f.y;
    v.z += h * f.z;
    x.x += R.dt * v.x;
    x.y += R.dt * v.y;
    x.z += R.dt * v.z;
    if (x.z > R.hz) {
      x.z = R.Lz - x.z;
      v.z = -v.z;
    } else if (x.z < -R.hz) {
      x.z = -R.Lz - x.z;
      v.z = -v.z;
    }
    if (x.x >= R.hx) x.x -= R.Lx;
    else if (x.x < -R.hx) x.x += R.Lx;
    if (x.y >= R.hy) x.y -= R.Ly;
    else if (x.y < -R.hy) x.y += R.Ly;
    const bool bad = !(fabs(x.x) <= R.hx && fabs(x.y) <= R.hy && fabs(x.z) <= R.hz);
    if (bad) atomicOr(a.status, kStatusUnstable);
    const dvec4 r0 = a.pos_ref[i];
    const double dx = wrap_diff(x.x - r0.x, R.Lx, R.hx);
    const double dy = wrap_diff(x.y - r0.y, R.Ly, R.hy);
    const double dz = x.z - r0.z;
    d2 = bad ? 0.0 : dx * dx + dy * dy + dz * dz;
    a.pos[i] = x;
    a.vel[i] = v;
    if (MIXED) a.lpos[i] = local_offset(R, x, a.home[i]);
  }
  unsigned long long b = (unsigned long long)__double_as_longlong(d2);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(kFull, b, o);
    b = t > b ? t : b;
  }
  if ((threadIdx.x & 31) == 0 && b) atomicMax(a.max_disp2, b);
}

// Fig. 3: v(t+dt) = v(t+dt/2) + a(t+dt) dt/2
__global__ void k_integrate_second(Arrays a, PotDev p) {
  if (halted(a)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  const RepDev& R = a.reps[a.rep[i]];
  dvec4 v = a.vel[i];
  const dvec4 f = a.frc[i];
  const double h = 0.5 * R.dt * p.inv_mass;
  v.x += h * f.x;
  v.y += h * f.y;
  v.z += h * f.z;
  a.vel[i] = v;
}

// ------------------------------------------------------------------------------------------------
// Fig. 4 (Berendsen): one block per replica reduces m sum v^2 in a fixed order on thermostat steps
__global__ void k_thermo_reduce(Arrays a, PotDev p) {
  if (halted(a)) return;
  const int r = blockIdx.x;
  const RepDev& R = a.reps[r];
  const long long s = *a.step;
  const bool act = R.n_th > 0 && R.n_vap > 0 && (s % R.n_th) == 0;
  if (!act) {
    if (threadIdx.x == 0) a.lambda[r] = 1.0;
    return;
  }
  double acc = 0.0;
  for (int k = threadIdx.x; k < R.n_vap; k += blockDim.x) {
    const dvec4 v = a.vel[R.vap_off + k];
    acc += v.x * v.x + v.y * v.y + v.z * v.z;
  }
  __shared__ double sh[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      const double T = p.mass * t / (3.0 * (double)R.n_vap);
      double lam = 1.0;
      if (T > 0.0) lam = sqrt(1.0 + R.lam_coef * (R.T0 / T - 1.0));
      a.lambda[r] = lam;
      *a.any_scale = 1;
    }
  }
}

__global__ void k_thermo_scale(Arrays a) {
  if (halted(a) || *a.any_scale == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  const double lam = a.lambda[a.rep[i]];
  dvec4 v = a.vel[i];
  v.x *= lam;
  v.y *= lam;
  v.z *= lam;
  a.vel[i] = v;
}

// ------------------------------------------------------------------------------------------------
// cell build: a counting sort of the vapour by cell, stable in the caller's molecule index

__global__ void k_cell_count(Arrays a, PotDev p, const int32_t* __restrict__ cell_rep) {
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  const RepDev& R = a.reps[a.rep[i]];
  const dvec4 x = a.pos[i];
  const int ix = cell_coord(x.x, R.hx, R.lcx, R.ncx);
  const int iy = cell_coord(x.y, R.hy, R.lcy, R.ncy);
  const int iz = cell_coord(x.z, R.hz, R.lcz, R.ncz);
  const int c = R.cell_off + (iz * R.ncy + iy) * R.ncx + ix;
  a.cell_tmp[i] = c;
  a.slot_tmp[i] = atomicAdd(&a.vcount[c], 1);
}

// exclusive scan of a 4096-element tile by 1024 threads; returns the tile total
__device__ int tile_exclusive_scan(const int32_t* in, int32_t* out, int n, int base) {
  __shared__ int warp_tot[32];
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
    int w = warp_tot[t];
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, wi, o);
      if (t >= o) wi += y;
    }
    warp_tot[t] = wi - w;  // exclusive prefix of warp totals
  }
  __syncthreads();
  int ex = warp_tot[t >> 5] + incl - run;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int idx = base + 4 * t + k;
    if (idx < n) out[idx] = ex;
    ex += v[k];
  }
  __shared__ int total;
  if (t == 1023) total = ex;
  __syncthreads();
  const int r = total;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(Arrays a, PotDev p) {
  if (halted(a) || !need_rebuild(a, p)) return;
  const int tot = tile_exclusive_scan(a.vcount, a.vstart, a.n_cells, blockIdx.x * 4096);
  if (threadIdx.x == 0) a.scan_tiles[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(Arrays a, PotDev p, int ntiles) {
  if (halted(a) || !need_rebuild(a, p)) return;
  tile_exclusive_scan(a.scan_tiles, a.scan_tiles, ntiles, 0);
}

__global__ void __launch_bounds__(1024) k_scan_add(Arrays a, PotDev p) {
  if (halted(a) || !need_rebuild(a, p)) return;
  const int add = a.scan_tiles[blockIdx.x];
  for (int k = threadIdx.x; k < 4096; k += blockDim.x) {
    const int idx = blockIdx.x * 4096 + k;
    if (idx < a.n_cells) a.vstart[idx] += add;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.vstart[a.n_cells] = a.n_total;
}

__global__ void k_scatter(Arrays a, PotDev p) {
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  a.perm_tmp[a.vstart[a.cell_tmp[i]] + a.slot_tmp[i]] = i;
}

// within a cell, molecules are ordered by their caller index: the sorted order depends only on
// the positions, not on the order in which atomics were served
__global__ void k_permute(Arrays a, PotDev p) {
  if (halted(a) || !need_rebuild(a, p)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_total) return;
  const int src = a.perm_tmp[s];
  const int c = a.cell_tmp[src];
  const int my_id = a.id[src];
  const int b = a.vstart[c], e = a.vstart[c + 1];
  int rank = 0;
  for (int t = b; t < e; ++t) rank += a.id[a.perm_tmp[t]] < my_id;
  const int dst = b + rank;
  const dvec4 x = a.pos[src];
  a.pos_alt[dst] = x;
  a.vel_alt[dst] = a.vel[src];
  a.frc_alt[dst] = a.frc[src];
  a.id_alt[dst] = my_id;
  const RepDev& R = a.reps[a.rep[src]];
  const int local = c - R.cell_off;
  const int ix = local % R.ncx, iy = (local / R.ncx) % R.ncy, iz = local / (R.ncx * R.ncy);
  const int home = pack_home(ix, iy, iz);
  a.home[dst] = home;
  a.pos_ref[dst] = x;
  a.lpos[dst] = local_offset(R, x, home);
}

__global__ void k_copyback(Arrays a, PotDev p) {
  if (halted(a) || !need_rebuild(a, p)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n_total) return;
  a.pos[i] = a.pos_alt[i];
  a.vel[i] = a.vel_alt[i];
  a.frc[i] = a.frc_alt[i];
  a.id[i] = a.id_alt[i];
}

// ------------------------------------------------------------------------------------------------
// Verlet-list build, one warp per cell. For each of the 27 neighbour cells the (molecule, candidate)
// pairs of the cell are spread over the 32 lanes; hits are appended to each molecule's list in
// (neighbour cell, candidate) order through a ballot/match prefix count, so lists are deterministic.
// Distances use the FP32 cell-local offsets; the list radius carries a margin above the FP32 error.

template <bool WALL>
__device__ __forceinline__ void list_pass(const Arrays& a, const PotDev& p, int i0, int nic,
                                          int j0, int nj, uint32_t code, float ox, float oy,
                                          float oz, int* cnt, int lane) {
  const float4* __restrict__ lj = WALL ? a.wlpos : a.lpos;
  uint32_t* __restrict__ out = WALL ? a.nbr_vw : a.nbr_vv;
  const int cap = WALL ? p.cap_vw : p.cap_vv;
  const int total = nic * nj;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = 0; base < total; base += 32) {
    const int q = base + lane;
    const bool valid = q < total;
    int il = 0, jl = 0;
    if (valid) {
      il = q / nj;
      jl = q - il * nj;
    }
    const int i = i0 + il, j = j0 + jl;
    bool hit = false;
    if (valid && (WALL || i != j)) {
      const float4 li = a.lpos[i];
      const float4 b = lj[j];
      const float dx = (li.x - b.x) - ox;
      const float dy = (li.y - b.y) - oy;
      const float dz = (li.z - b.z) - oz;
      hit = dx * dx + dy * dy + dz * dz < p.rl2f;
    }
    const unsigned hits = __ballot_sync(kFull, hit);
    const unsigned same = __match_any_sync(kFull, valid ? il : 64 + lane);
    if (hit) {
      const int slot = cnt[il] + __popc(hits & same & lt);
      if (slot < cap) out[(size_t)slot * a.n_total + i] = (uint32_t)j | code;
    }
    __syncwarp();
    if (valid && (same & lt) == 0) cnt[il] += __popc(hits & same);
    __syncwarp();
  }
}

__global__ void k_list_build(Arrays a, PotDev p, const int32_t* __restrict__ cell_rep) {
  if (halted(a) || !need_rebuild(a, p)) return;
  extern __shared__ int sh_cnt[];
  const int warp_in_block = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp_in_block;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.n_rebuilds, 1ull);
  if (c >= a.n_cells) return;
  int* cnt_vv = sh_cnt + warp_in_block * 64;
  int* cnt_vw = cnt_vv + 32;
  const int i_begin = a.vstart[c], i_end = a.vstart[c + 1];
  if (lane == 0) a.vcount[c] = 0;  // ready for the next build
  if (i_end == i_begin) return;
  const RepDev& R = a.reps[cell_rep[c]];
  const int local = c - R.cell_off;
  const int ix = local % R.ncx, iy = (local / R.ncx) % R.ncy, iz = local / (R.ncx * R.ncy);
  int max_vv = 0, max_vw = 0;
  for (int i0 = i_begin; i0 < i_end; i0 += 32) {
    const int nic = min(32, i_end - i0);
    cnt_vv[lane] = 0;
    cnt_vw[lane] = 0;
    __syncwarp();
    for (int dz = -1; dz <= 1; ++dz) {
      const int jz = iz + dz;
      if (jz < 0 || jz >= R.ncz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int jy = (iy + dy + R.ncy) % R.ncy;
        for (int dx = -1; dx <= 1; ++dx) {
          const int jx = (ix + dx + R.ncx) % R.ncx;
          const int cn = R.cell_off + (jz * R.ncy + jy) * R.ncx + jx;
          const uint32_t code = ((uint32_t)(dx + 1) << 26) | ((uint32_t)(dy + 1) << 28) |
                                ((uint32_t)(dz + 1) << 30);
          const float ox = dx * R.lcxf, oy = dy * R.lcyf, oz = dz * R.lczf;
          const int vj0 = a.vstart[cn], vj1 = a.vstart[cn + 1];
          if (vj1 > vj0)
            list_pass<false>(a, p, i0, nic, vj0, vj1 - vj0, code, ox, oy, oz, cnt_vv, lane);
          const int wj0 = a.wstart[cn], wj1 = a.wstart[cn + 1];
          if (wj1 > wj0)
            list_pass<true>(a, p, i0, nic, wj0, wj1 - wj0, code, ox, oy, oz, cnt_vw, lane);
        }
      }
    }
    if (lane < nic) {
      const int nv = cnt_vv[lane], nw = cnt_vw[lane];
      if (nv > p.cap_vv || nw > p.cap_vw) atomicOr(a.status, kStatusOverflow);
      a.n_vv[i0 + lane] = min(nv, p.cap_vv);
      a.n_vw[i0 + lane] = min(nw, p.cap_vw);
      max_vv = max(max_vv, nv);
      max_vw = max(max_vw, nw);
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    max_vv = max(max_vv, __shfl_xor_sync(kFull, max_vv, o));
    max_vw = max(max_vw, __shfl_xor_sync(kFull, max_vw, o));
  }
  if (lane == 0) {
    atomicMax(a.max_nvv, max_vv);
    atomicMax(a.max_nvw, max_vw);
  }
}

// ------------------------------------------------------------------------------------------------
// Pair forces (Eq. 2, Fig. 1): f_i = sum_j F(r_ij)/r_ij * (r_i - r_j) over list entries with
// r^2 < rc^2, F(r)/r = inv2 * inv6 * (48 eps s^12 inv6 - 24 eps s^6), inv2 = 1/r^2, inv6 = inv2^3.
// The vapour list is full (each pair held by both molecules), so each molecule's force is a sum
// it owns: no atomics, the result does not depend on scheduling.
//
// FP64 variant: everything in FP64.

template <bool STATS>
__global__ void k_forces_fp64(Arrays a, PotDev p) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.max_disp2 = 0ull;
    *a.force_rebuild = 0;
  }
  if (halted(a)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < a.n_total;
  int cnt = 0;
  if (live) {
    const RepDev& R = a.reps[a.rep[i]];
    const dvec4 xi = a.pos[i];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    double pe = 0.0, vir = 0.0, pew = 0.0, virw = 0.0, d2w = __longlong_as_double(0x7ff0000000000000ll);
    int cvw = 0;
    const int nv = a.n_vv[i];
    const uint32_t* __restrict__ lv = a.nbr_vv + i;
    for (int k = 0; k < nv; ++k) {
      const int j = (int)(lv[(size_t)k * a.n_total] & kIndexMask);
      const dvec4 xj = a.pos[j];
      const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
      const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
      const double dz = xi.z - xj.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < p.rc2) {
        const double inv2 = 1.0 / r2;
        const double inv6 = inv2 * inv2 * inv2;
        const double fr = inv2 * inv6 * fma(p.a12, inv6, -p.b6);
        fx = fma(fr, dx, fx);
        fy = fma(fr, dy, fy);
        fz = fma(fr, dz, fz);
        ++cnt;
        if (STATS) {
          pe += 0.5 * (inv6 * fma(p.e12, inv6, -p.e6) - p.ushift);
          vir += 0.5 * fr * r2;
        }
      }
    }
    const int nw = a.n_vw[i];
    const uint32_t* __restrict__ lw = a.nbr_vw + i;
    for (int k = 0; k < nw; ++k) {
      const int j = (int)(lw[(size_t)k * a.n_total] & kIndexMask);
      const dvec4 xj = a.wpos[j];
      const double dx = image_hi(xi.x - xj.x, R.Lx, R.hi_thr_x);
      const double dy = image_hi(xi.y - xj.y, R.Ly, R.hi_thr_y);
      const double dz = xi.z - xj.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < p.rcw2) {
        const double inv2 = 1.0 / r2;
        const double inv6 = inv2 * inv2 * inv2;
        const double fr = inv2 * inv6 * fma(p.a12w, inv6, -p.b6w);
        fx = fma(fr, dx, fx);
        fy = fma(fr, dy, fy);
        fz = fma(fr, dz, fz);
        ++cvw;
        if (STATS) {
          pew += inv6 * fma(p.e12w, inv6, -p.e6w) - p.ushift_w;
          virw += fr * r2;
          d2w = fmin(d2w, r2);
        }
      }
    }
    a.frc[i] = make_dvec4(fx, fy, fz, 0.0);
    if (STATS) {
      a.pe_i[i] = pe;
      a.pevw_i[i] = pew;
      a.vir_i[i] = vir;
      a.virw_i[i] = virw;
      a.d2w_i[i] = d2w;
      a.cnt_vv_i[i] = cnt;
      a.cnt_vw_i[i] = cvw;
    }
    cnt += 2 * cvw;  // vapour pairs are seen from both ends: count twice, halve at read-out
  }
  if (!STATS) {
    unsigned long long c = warp_sum((unsigned long long)cnt);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.pair_count, c);
  }
}

// Mixed variant: pair terms in FP32 from the cell-local FP32 offsets (the displacement is
// (l_i - l_j) - dc * cell side, all terms small, so the FP32 rounding is relative to the cell size
// rather than the box), per-molecule sums in compensated FP32 (TwoSum), written as FP64.
// Energies and virials of the observable pass are accumulated in FP64.

template <bool STATS>
__global__ void k_forces_mixed(Arrays a, PotDev p) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.max_disp2 = 0ull;
    *a.force_rebuild = 0;
  }
  if (halted(a)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < a.n_total;
  int cnt = 0;
  if (live) {
    const RepDev& R = a.reps[a.rep[i]];
    const float4 li = a.lpos[i];
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    double pe = 0.0, vir = 0.0, pew = 0.0, virw = 0.0, d2w = __longlong_as_double(0x7ff0000000000000ll);
    int cvw = 0;
    const int nv = a.n_vv[i];
    const uint32_t* __restrict__ lv = a.nbr_vv + i;
    for (int k = 0; k < nv; ++k) {
      const uint32_t e = lv[(size_t)k * a.n_total];
      const float4 b = a.lpos[e & kIndexMask];
      const float dx = (li.x - b.x) - (float)((int)((e >> 26) & 3u) - 1) * R.lcxf;
      const float dy = (li.y - b.y) - (float)((int)((e >> 28) & 3u) - 1) * R.lcyf;
      const float dz = (li.z - b.z) - (float)((int)(e >> 30) - 1) * R.lczf;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < p.rc2f) {
        const float inv2 = __frcp_rn(r2);
        const float inv6 = inv2 * inv2 * inv2;
        const float fr = inv2 * inv6 * fmaf(p.a12f, inv6, -p.b6f);
        two_sum_acc(sx, cx, fr * dx);
        two_sum_acc(sy, cy, fr * dy);
        two_sum_acc(sz, cz, fr * dz);
        ++cnt;
        if (STATS) {
          pe += 0.5 * ((double)(inv6 * fmaf(p.e12f, inv6, -p.e6f)) - p.ushift);
          vir += 0.5 * (double)(fr * r2);
        }
      }
    }
    const int nw = a.n_vw[i];
    const uint32_t* __restrict__ lw = a.nbr_vw + i;
    for (int k = 0; k < nw; ++k) {
      const uint32_t e = lw[(size_t)k * a.n_total];
      const float4 b = a.wlpos[e & kIndexMask];
      const float dx = (li.x - b.x) - (float)((int)((e >> 26) & 3u) - 1) * R.lcxf;
      const float dy = (li.y - b.y) - (float)((int)((e >> 28) & 3u) - 1) * R.lcyf;
      const float dz = (li.z - b.z) - (float)((int)(e >> 30) - 1) * R.lczf;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < p.rcw2f) {
        const float inv2 = __frcp_rn(r2);
        const float inv6 = inv2 * inv2 * inv2;
        const float fr = inv2 * inv6 * fmaf(p.a12wf, inv6, -p.b6wf);
        two_sum_acc(sx, cx, fr * dx);
        two_sum_acc(sy, cy, fr * dy);
        two_sum_acc(sz, cz, fr * dz);
        ++cvw;
        if (STATS) {
          pew += (double)(inv6 * fmaf(p.e12wf, inv6, -p.e6wf)) - p.ushift_w;
          virw += (double)(fr * r2);
          d2w = fmin(d2w, (double)r2);
        }
      }
    }
    a.frc[i] = make_dvec4((double)sx + (double)cx, (double)sy + (double)cy,
                            (double)sz + (double)cz, 0.0);
    if (STATS) {
      a.pe_i[i] = pe;
      a.pevw_i[i] = pew;
      a.vir_i[i] = vir;
      a.virw_i[i] = virw;
      a.d2w_i[i] = d2w;
      a.cnt_vv_i[i] = cnt;
      a.cnt_vw_i[i] = cvw;
    }
    cnt += 2 * cvw;
  }
  if (!STATS) {
    unsigned long long c = warp_sum((unsigned long long)cnt);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.pair_count, c);
  }
}

// ------------------------------------------------------------------------------------------------
// observables: pore assignment, occupancy, adsorbed count, axial profile (integer atomics: exact)

__global__ void k_observe(Arrays a, PotDev p) {
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

// per-replica sums in a fixed order (one block per replica): ke, pe_vv, pe_vw, vir_vv, vir_vw,
// ordered vapour pair count, wall pair count
__global__ void k_rep_sums(Arrays a, PotDev p) {
  const int r = blockIdx.x;
  const RepDev& R = a.reps[r];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int k = threadIdx.x; k < R.n_vap; k += blockDim.x) {
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
  __shared__ double sh[7][32];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const double w = warp_sum(acc[q]);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      double t = threadIdx.x < (blockDim.x >> 5) ? sh[q][threadIdx.x] : 0.0;
      t = warp_sum(t);
      if (threadIdx.x == 0) a.rep_sums[r * 8 + q] = (q == 0 ? 0.5 * p.mass * t : t);
    }
  }
}

inline int nblocks(long long n, int b) { return n > 0 ? (int)((n + b - 1) / b) : 1; }

}  // namespace

// ------------------------------------------------------------------------------------------------
// launchers

void launch_integrate_first(const Arrays& a, const PotDev& p, bool mixed, cudaStream_t s) {
  const int b = 256;
  if (mixed)
    k_integrate_first<true><<<nblocks(a.n_total, b), b, 0, s>>>(a, p);
  else
    k_integrate_first<false><<<nblocks(a.n_total, b), b, 0, s>>>(a, p);
}

void launch_rebuild(const Arrays& a, const PotDev& p, const Tuning& t, const int32_t* cell_rep,
                    cudaStream_t s) {
  const int b = 256;
  const int nt = nblocks(a.n_total, b);
  const int ntiles = nblocks(a.n_cells, 4096);
  k_cell_count<<<nt, b, 0, s>>>(a, p, cell_rep);
  k_scan_tiles<<<ntiles, 1024, 0, s>>>(a, p);
  k_scan_top<<<1, 1024, 0, s>>>(a, p, ntiles);
  k_scan_add<<<ntiles, 1024, 0, s>>>(a, p);
  k_scatter<<<nt, b, 0, s>>>(a, p);
  k_permute<<<nt, b, 0, s>>>(a, p);
  k_copyback<<<nt, b, 0, s>>>(a, p);
  const int lb = t.list_block;
  const int warps = lb / 32;
  k_list_build<<<nblocks(a.n_cells, warps), lb, warps * 64 * sizeof(int), s>>>(a, p, cell_rep);
}

void launch_forces(const Arrays& a, const PotDev& p, bool mixed, bool stats, const Tuning& t,
                   cudaStream_t s) {
  const int b = t.force_block;
  const int g = nblocks(a.n_total, b);
  if (mixed) {
    if (stats) k_forces_mixed<true><<<g, b, 0, s>>>(a, p);
    else k_forces_mixed<false><<<g, b, 0, s>>>(a, p);
  } else {
    if (stats) k_forces_fp64<true><<<g, b, 0, s>>>(a, p);
    else k_forces_fp64<false><<<g, b, 0, s>>>(a, p);
  }
}

void launch_integrate_second(const Arrays& a, const PotDev& p, cudaStream_t s) {
  const int b = 256;
  k_integrate_second<<<nblocks(a.n_total, b), b, 0, s>>>(a, p);
}

void launch_thermostat(const Arrays& a, const PotDev& p, cudaStream_t s) {
  k_thermo_reduce<<<a.n_reps, 256, 0, s>>>(a, p);
  const int b = 256;
  k_thermo_scale<<<nblocks(a.n_total, b), b, 0, s>>>(a);
}

void launch_observables(const Arrays& a, const PotDev& p, cudaStream_t s) {
  const int b = 256;
  k_observe<<<nblocks(a.n_total, b), b, 0, s>>>(a, p);
  k_rep_sums<<<a.n_reps, 256, 0, s>>>(a, p);
}

int kernels_per_step() { return 1 + 8 + 1 + 1 + 2; }
int kernels_per_rebuild() { return 8; }

}  // namespace mdk
