// md_noalloc.cu -- md_forces_noalloc: FP64 Lennard-Jones forces on caller-owned device arrays that
// allocate no memory. The cell list it needs lives in one fixed-size scratch array in this file.
//
// Why: some callers cannot call cudaMalloc/cudaFree -- an application that has handed (nearly) all
// device memory to its own pool allocator, where a further cudaMalloc fails or fragments that pool,
// or a latency-critical host thread that must not hit the implicit device synchronisation cudaFree
// performs. They pass their own inputs and outputs; the scratch below is reserved once, when the
// library is loaded, and held on every GPU until the process exits.
//
// Limits: n_vapor + n_wall <= kNaMaxAtoms and at most kNaMaxCells cells of side >= max(rc, rc_w)
// (at least 3 across x and y). Every call reuses the same scratch: calls that overlap on the GPU
// (on different streams, or from different host threads) race with each other and must not.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/md.h"

namespace {

constexpr int kNaMaxAtoms = 1 << 18;
constexpr int kNaMaxCells = 1 << 16;
constexpr size_t kNaInts = 2 * (size_t)kNaMaxCells + 2 * ((size_t)kNaMaxCells + 1) +
                           3 * (size_t)kNaMaxAtoms;
constexpr int kNaMaxDevices = 64;

// device scratch (int32): cnt_v, cnt_w [cells]; start_v, start_w [cells + 1];
// cell id, slot, sorted index [atoms]
static __device__ __align__(256) int32_t g_na_scratch[kNaInts];

std::mutex g_na_mutex;
int32_t* g_na_ptr[kNaMaxDevices] = {};

struct NaGeom {
  double Lx, Ly, Lz, hx, hy, hz, lx, ly, lz;
  int nx, ny, nz, ncell, n, nw;
  double rc2, rcw2, a12, b6, a12w, b6w;
};

struct NaScratch {
  int32_t *cnt_v, *cnt_w, *start_v, *start_w, *cell, *slot, *sorted;
};

NaScratch carve(int32_t* s) {
  NaScratch p;
  p.cnt_v = s;
  p.cnt_w = p.cnt_v + kNaMaxCells;
  p.start_v = p.cnt_w + kNaMaxCells;
  p.start_w = p.start_v + (kNaMaxCells + 1);
  p.cell = p.start_w + (kNaMaxCells + 1);
  p.slot = p.cell + kNaMaxAtoms;
  p.sorted = p.slot + kNaMaxAtoms;
  return p;
}

__device__ __forceinline__ int na_coord(double u, double half, double l, int nc) {
  int c = (int)floor((u + half) / l);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// periodic wrap of an x or y coordinate into [-L/2, L/2); a coordinate already inside is returned
// unchanged (bit for bit), so in-box inputs give the same cells and distances as without the wrap
__device__ __forceinline__ double na_wrap(double u, double L, double half) {
  if (u >= half || u < -half) u -= L * floor((u + half) / L);
  return u;
}

// cell of a point: x and y wrapped periodically first, z (walls at +-Lz/2) clamped into the grid
__device__ __forceinline__ int na_cell(const NaGeom& g, const double* p) {
  const int ix = na_coord(na_wrap(p[0], g.Lx, g.hx), g.hx, g.lx, g.nx);
  const int iy = na_coord(na_wrap(p[1], g.Ly, g.hy), g.hy, g.ly, g.ny);
  const int iz = na_coord(p[2], g.hz, g.lz, g.nz);
  return (iz * g.ny + iy) * g.nx + ix;
}

__device__ __forceinline__ double na_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

// counts must start at zero: the previous call left its counts in the shared scratch
__global__ void k_na_clear(NaScratch s, int ncell) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    s.cnt_v[c] = 0;
    s.cnt_w[c] = 0;
  }
}

__global__ void k_na_count(NaScratch s, NaGeom g, const double* __restrict__ x,
                           const double* __restrict__ w) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.n + g.nw) return;
  const bool wall = a >= g.n;
  const double* p = wall ? w + 3 * (size_t)(a - g.n) : x + 3 * (size_t)a;
  const int c = na_cell(g, p);
  s.cell[a] = c;
  s.slot[a] = atomicAdd(wall ? &s.cnt_w[c] : &s.cnt_v[c], 1);
}

// exclusive scans of both count arrays by one block of 1024 threads, tile by tile
__global__ void __launch_bounds__(1024) k_na_scan(NaScratch s, int ncell) {
  __shared__ int warp_tot[32];
  __shared__ int carry_sh;
  for (int which = 0; which < 2; ++which) {
    const int32_t* in = which ? s.cnt_w : s.cnt_v;
    int32_t* out = which ? s.start_w : s.start_v;
    int carry = 0;
    for (int base = 0; base < ncell; base += 1024) {
      const int idx = base + threadIdx.x;
      const int v = idx < ncell ? in[idx] : 0;
      int incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((threadIdx.x & 31) >= o) incl += y;
      }
      if ((threadIdx.x & 31) == 31) warp_tot[threadIdx.x >> 5] = incl;
      __syncthreads();
      if (threadIdx.x < 32) {
        const int t = warp_tot[threadIdx.x];
        int ti = t;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, ti, o);
          if ((int)threadIdx.x >= o) ti += y;
        }
        warp_tot[threadIdx.x] = ti - t;
        if (threadIdx.x == 31) carry_sh = ti;
      }
      __syncthreads();
      if (idx < ncell) out[idx] = carry + warp_tot[threadIdx.x >> 5] + incl - v;
      carry += carry_sh;
      __syncthreads();
    }
    if (threadIdx.x == 0) out[ncell] = carry;
  }
}

__global__ void k_na_scatter(NaScratch s, NaGeom g) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= g.n + g.nw) return;
  if (a < g.n)
    s.sorted[s.start_v[s.cell[a]] + s.slot[a]] = a;
  else
    s.sorted[g.n + s.start_w[s.cell[a]] + s.slot[a]] = a - g.n;
}

// one thread per vapour molecule: all molecules and wall atoms of the 27 surrounding cells
__global__ void k_na_forces(NaScratch s, NaGeom g, const double* __restrict__ x,
                            const double* __restrict__ w, double* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const double xi = na_wrap(x[3 * (size_t)i], g.Lx, g.hx);
  const double yi = na_wrap(x[3 * (size_t)i + 1], g.Ly, g.hy), zi = x[3 * (size_t)i + 2];
  const int c = s.cell[i];
  const int ix = c % g.nx, iy = (c / g.nx) % g.ny, iz = c / (g.nx * g.ny);
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int jz = iz + dz;
    if (jz < 0 || jz >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int jy = (iy + dy + g.ny) % g.ny;
      for (int dx = -1; dx <= 1; ++dx) {
        const int jx = (ix + dx + g.nx) % g.nx;
        const int cn = (jz * g.ny + jy) * g.nx + jx;
        for (int k = s.start_v[cn]; k < s.start_v[cn + 1]; ++k) {
          const int j = s.sorted[k];
          if (j == i) continue;
          const double ddx = na_image(xi - na_wrap(x[3 * (size_t)j], g.Lx, g.hx), g.Lx);
          const double ddy = na_image(yi - na_wrap(x[3 * (size_t)j + 1], g.Ly, g.hy), g.Ly);
          const double ddz = zi - x[3 * (size_t)j + 2];
          const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
          if (r2 < g.rc2) {
            const double inv2 = 1.0 / r2, inv6 = inv2 * inv2 * inv2;
            const double fr = inv2 * inv6 * fma(g.a12, inv6, -g.b6);
            fx = fma(fr, ddx, fx);
            fy = fma(fr, ddy, fy);
            fz = fma(fr, ddz, fz);
          }
        }
        for (int k = s.start_w[cn]; k < s.start_w[cn + 1]; ++k) {
          const int j = s.sorted[g.n + k];
          const double ddx = na_image(xi - na_wrap(w[3 * (size_t)j], g.Lx, g.hx), g.Lx);
          const double ddy = na_image(yi - na_wrap(w[3 * (size_t)j + 1], g.Ly, g.hy), g.Ly);
          const double ddz = zi - w[3 * (size_t)j + 2];
          const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
          if (r2 < g.rcw2) {
            const double inv2 = 1.0 / r2, inv6 = inv2 * inv2 * inv2;
            const double fr = inv2 * inv6 * fma(g.a12w, inv6, -g.b6w);
            fx = fma(fr, ddx, fx);
            fy = fma(fr, ddy, fy);
            fz = fma(fr, ddz, fz);
          }
        }
      }
    }
  }
  f[3 * (size_t)i] = fx;
  f[3 * (size_t)i + 1] = fy;
  f[3 * (size_t)i + 2] = fz;
}

md_status na_fail(char* err, int32_t err_len, const char* msg) {
  if (err && err_len > 0) {
    std::strncpy(err, msg, (size_t)err_len - 1);
    err[err_len - 1] = '\0';
  }
  return MD_EINVAL;
}

// device address of the scratch array on the current device, looked up once per device
md_status na_scratch_ptr(int32_t** out, char* err, int32_t err_len) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    if (err && err_len > 0) na_fail(err, err_len, "no usable current CUDA device");
    return MD_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      if (err && err_len > 0) na_fail(err, err_len, "cudaGetSymbolAddress of the scratch failed");
      return MD_ECUDA;
    }
    g_na_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_na_ptr[dev];
  return MD_OK;
}

}  // namespace

extern "C" md_status md_forces_noalloc(const md_potential* pot, double Lx, double Ly, double Lz,
                                       const double* d_x, int64_t n_vapor, const double* d_wall,
                                       int64_t n_wall, double* d_f, void* stream, char* err,
                                       int32_t err_len) {
  if (err && err_len > 0) err[0] = '\0';
  if (!pot) return na_fail(err, err_len, "potential is NULL");
  // the same rules (and message) as md_create for the fields this entry point reads
  for (double q : {pot->eps, pot->sigma, pot->mass, pot->rc, pot->eps_w, pot->sigma_w, pot->rc_w})
    if (!std::isfinite(q)) return na_fail(err, err_len, "potential: a parameter is not finite");
  if (!(pot->sigma > 0 && pot->sigma_w > 0 && pot->rc > 0 && pot->rc_w > 0))
    return na_fail(err, err_len, "sigma, sigma_w, rc, rc_w must be > 0");
  if (!(std::isfinite(Lx) && std::isfinite(Ly) && std::isfinite(Lz)))
    return na_fail(err, err_len, "box: a side is not finite");
  if (!(Lx > 0 && Ly > 0 && Lz > 0)) return na_fail(err, err_len, "box must be positive");
  if (n_vapor < 0 || n_wall < 0) return na_fail(err, err_len, "negative count");
  if ((n_vapor > 0 && (!d_x || !d_f)) || (n_wall > 0 && !d_wall))
    return na_fail(err, err_len, "NULL device array");
  if (n_vapor + n_wall > kNaMaxAtoms) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "n_vapor + n_wall = %lld exceeds the no-alloc limit of %d atoms",
                  (long long)(n_vapor + n_wall), kNaMaxAtoms);
    return na_fail(err, err_len, msg);
  }
  const double rcut = pot->rc > pot->rc_w ? pot->rc : pot->rc_w;
  if (Lx / rcut > kNaMaxCells || Ly / rcut > kNaMaxCells || Lz / rcut > kNaMaxCells)
    return na_fail(err, err_len, "box too large for the no-alloc cell limit");
  NaGeom g;
  g.nx = (int)(Lx / rcut);
  g.ny = (int)(Ly / rcut);
  g.nz = (int)(Lz / rcut);
  if (g.nz < 1) g.nz = 1;
  if (g.nx < 3 || g.ny < 3)
    return na_fail(err, err_len, "box x/y must hold at least 3 cells of max(rc, rc_w)");
  if ((long long)g.nx * g.ny * g.nz > kNaMaxCells) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "%lld cells exceed the no-alloc limit of %d cells",
                  (long long)g.nx * g.ny * g.nz, kNaMaxCells);
    return na_fail(err, err_len, msg);
  }
  if (n_vapor == 0) return MD_OK;
  int32_t* base = nullptr;
  md_status st = na_scratch_ptr(&base, err, err_len);
  if (st != MD_OK) return st;
  g.Lx = Lx; g.Ly = Ly; g.Lz = Lz;
  g.hx = 0.5 * Lx; g.hy = 0.5 * Ly; g.hz = 0.5 * Lz;
  g.lx = Lx / g.nx; g.ly = Ly / g.ny; g.lz = Lz / g.nz;
  g.ncell = g.nx * g.ny * g.nz;
  g.n = (int)n_vapor;
  g.nw = (int)n_wall;
  const double s6 = pot->sigma * pot->sigma * pot->sigma * pot->sigma * pot->sigma * pot->sigma;
  const double w6 = pot->sigma_w * pot->sigma_w * pot->sigma_w * pot->sigma_w * pot->sigma_w *
                    pot->sigma_w;
  g.rc2 = pot->rc * pot->rc;
  g.rcw2 = pot->rc_w * pot->rc_w;
  g.a12 = 48.0 * pot->eps * s6 * s6;
  g.b6 = 24.0 * pot->eps * s6;
  g.a12w = 48.0 * pot->eps_w * w6 * w6;
  g.b6w = 24.0 * pot->eps_w * w6;
  const NaScratch s = carve(base);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  // an error left by the caller's own earlier work stays theirs: report it without clearing it,
  // so that the error read after the launches below is this call's
  const cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) {
    if (err && err_len > 0) {
      char msg[200];
      std::snprintf(msg, sizeof msg, "a CUDA error was pending before this call (left set): %s",
                    cudaGetErrorString(pending));
      na_fail(err, err_len, msg);
    }
    return MD_ECUDA;
  }
  const int atoms = g.n + g.nw;
  k_na_clear<<<(g.ncell + 255) / 256, 256, 0, cs>>>(s, g.ncell);
  k_na_count<<<(atoms + 255) / 256, 256, 0, cs>>>(s, g, d_x, d_wall);
  k_na_scan<<<1, 1024, 0, cs>>>(s, g.ncell);
  k_na_scatter<<<(atoms + 255) / 256, 256, 0, cs>>>(s, g);
  k_na_forces<<<(g.n + 127) / 128, 128, 0, cs>>>(s, g, d_x, d_wall, d_f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (err && err_len > 0) na_fail(err, err_len, cudaGetErrorString(e));
    return MD_ECUDA;
  }
  return MD_OK;
}
