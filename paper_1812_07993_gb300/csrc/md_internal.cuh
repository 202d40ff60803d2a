// md_internal.cuh -- device data layout and kernel entry points of the pore / water-vapour MD
// library (arXiv:1812.07993, Sec. 2-3). Internal to the library; the public ABI is include/md.h.
//
// Layout in HBM (all replicas of a context packed back to back):
//   vapour, in cell-sorted order (re-sorted at every list build):
//     pos, vel, frc   32-byte aligned double4 (x, y, z, unused): one 256-bit access per molecule
//     lpos            float4, position relative to the centre of the home cell (FP32 staging for the
//                     list build, the screens and the mixed-precision pair kernels)
//     lref            float4, lpos at the last list build (the skin check: the displacement since
//                     then is lpos - lref, both from the same centre)
//     lpos_lo         float4, that offset minus lpos, rounded to FP32: with lpos the double-float
//                     offset of the double-float pair kernels
//     home, id, rep   int32: home cell (packed ix | iy << 10 | iz << 20), caller index within the
//                     replica, replica
//     nbr             Verlet list, one row of `cap` slots per molecule: partners j > i then wall
//                     atoms from the front (vapour first), partners j < i from the back;
//                     n_front / n_back / n_vh give the lengths (n_vh: vapour part of the front)
//     order           optional processing order: molecules sorted by list length, longest first
//   FP64 pair path (Newton's third law, deterministic):
//     fwd             for each front vapour slot of a molecule, the pairbuf entry
//                     partner * cap_v + (its back slot) that receives the pair force
//     pairbuf         forces of the pairs held by lower partners, [molecule * cap_v + back slot],
//                     plus one spare entry at the end
//     fpart           partial force of the half-list pass
//   flat stream (force_tpp 64, allocated on first use): flat_ent / flat_own, the front rows of all
//     molecules in cell order, copied at every rebuild
//   wall (static, sorted by cell once at creation): wpos double4, wlpos and wlpos_lo float4,
//     wstart (CSR)
//   cells: per-replica grids of side >= max(rc, rc_w) + skin, at least 3 across x and y.
// A list entry packs the neighbour index in the low 26 bits -- a vapour molecule below n_total, a
// wall atom at n_total + its index -- and the neighbour's home-cell offset relative to the
// molecule's home cell, 2 bits per axis (value + 1), in bits 26-31.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "md_fpconv.cuh"

namespace mdk {

// 32-byte aligned FP64 vector: one 256-bit load/store per molecule record
using dvec4 = double4_32a;
__host__ __device__ inline dvec4 make_dvec4(double x, double y, double z, double w) {
  return make_double4_32a(x, y, z, w);
}

constexpr uint32_t kIndexBits = 26;
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
constexpr int kMaxIndex = (1 << kIndexBits) - 1;
constexpr int kMaxCap = 1023;  // longest list (vapour + wall neighbours) a molecule may hold

// pair-term precision of a kernel (the values of md_precision)
constexpr int kPrecFP64 = 0;
constexpr int kPrecMixed = 1;
constexpr int kPrecDF64 = 2;
// force_tpp of the flat stream: a chunk's rows screened as one stream of entries (atomic form)
constexpr int kFlatTpp = 64;
constexpr int kFlatPerMol = 128;  // the flat stream's capacity per molecule (at most the row's)
constexpr int kFlatBlock = 1024;  // molecules per block of the stream's fill

// sticky device status bits
constexpr int kStatusOverflow = 1;
constexpr int kStatusUnstable = 2;
constexpr int kStatusTimeout = 4;
constexpr int kStatusBounds = 8;   // an index check of the checked build failed

// Index checks of the checked build (compiled with -DMD_CHECKED): an index read from device data
// (a list entry, the processing order, a pair slot, a cell or sort index) that lies outside
// [0, lim) sets the sticky status bit kStatusBounds and is replaced by 0, so the access stays
// inside its array and the run reports MD_EBOUNDS instead of trapping. In the normal build the
// check is the index itself.
// The first failing check records its source line (status[1]) for md_last_error.
#ifdef MD_CHECKED
__device__ __forceinline__ long long chk_index(int32_t* status, long long idx, long long lim,
                                               int line) {
  if (idx >= 0 && idx < lim) return idx;
  atomicOr(status, kStatusBounds);
  atomicCAS(status + 1, 0, line);
  return 0;
}
#define MD_CHK(a, idx, lim)                                                                  \
  ((typename std::decay<decltype(idx)>::type)::mdk::chk_index((a).status, (long long)(idx),    \
                                                               (long long)(lim), __LINE__))
#else
#define MD_CHK(a, idx, lim) (idx)
#endif

struct RepDev {
  double Lx, Ly, Lz, hx, hy, hz;
  double T0, dt, lam_coef;          // lam_coef = n_th dt / tau_B
  double slab_half;
  double lcx, lcy, lcz;             // cell sides
  double ilcx, ilcy, ilcz;          // and their inverses (the device's cell assignment)
  double bin_width;
  float lcxf, lcyf, lczf;
  uint32_t hi_thr_x, hi_thr_y;      // high word of L/2: |d| above it needs the periodic image
  int32_t n_th;
  int32_t vap_off, n_vap;
  int32_t wall_off, n_wall;
  int32_t cell_off, ncx, ncy, ncz;
  int32_t pore_off, n_pores;
  int32_t group_off, n_groups;      // adsorbed counters / profile rows
  int32_t n_bins;
  int32_t prof_off;                 // first profile counter of this replica
  double half_dt_m, dt_m;           // dt/(2m) and dt/m
  int32_t ctr_off;                  // this replica's cell centres in cell_ctr: x, then y, then z
  int32_t dims;                     // 3, or 2 for a planar system (temperature with 2N)
  int32_t hard;                     // 1: hard reflecting walls (no wall atoms)
  float lcx_lo, lcy_lo, lcz_lo;     // cell sides minus their FP32 roundings (double-float form)
};

struct PoreDev {
  int32_t kind;
  double cx, cy, r0, r1, r_cavity, width;
  double vol;                       // volume of the carved region inside the slab
};

struct PotDev {
  double rc2, rcw2;
  double a12, b6, a12w, b6w;        // force:  F/r = inv2 * inv6 * (a12 * inv6 - b6)
  double e12, e6, e12w, e6w;        // energy: U = inv6 * (e12 * inv6 - e6)
  double ushift, ushift_w;
  double inv_mass, mass;
  double half_skin2;                // rebuild when a displacement^2 reaches this
  double group_disp2;               // with a rebuild under way, replicas past this rebuild too
  double r_ads2;
  float rc2f, rcw2f, rl2f;          // FP32 cutoffs and the (padded) list radius^2
  float rc2f_lo, rc2f_hi, rcw2f_lo, rcw2f_hi;  // FP32 band around the cutoff decided in FP64
  float a12f, b6f, a12wf, b6wf, e12f, e6f, e12wf, e6wf;
  float a12l, b6l, a12wl, b6wl;     // force constants minus their FP32 roundings (double-float)
  int32_t cap;                      // list capacity per molecule (vapour + wall)
  int32_t cap_v;                    // vapour half-pair / reverse capacity per molecule
};

// Device pointers of one context (passed by value to kernels).
struct Arrays {
  dvec4 *pos, *vel, *frc;
  dvec4 *pos_alt, *vel_alt, *frc_alt;
  float4* lpos;
  float4* lpos_lo;                  // double-float pair terms: lpos's remainder, offset - lpos
  float4* lref;                     // lpos at the last list build (skin check)
  int32_t *home, *id, *rep, *id_alt;
  int32_t *cell_tmp, *slot_tmp, *perm_tmp;
  uint32_t* nbr;                    // [molecule * cap + slot]: front (j > i, walls), back (j < i)
  int32_t *n_front, *n_back, *n_vh; // front / back lengths; vapour entries at the front
  // optional processing order (longest list first)
  int32_t *order, *hist, *hstart;
  // the flat stream (force_tpp 64): the front rows in one array, filled at each rebuild once
  // allocated (NULL until then): entry k is list entry flat_ent[k] of molecule flat_own[k]
  uint32_t* flat_ent;
  int32_t* flat_own;
  int32_t* flat_part;               // entries per block of the fill
  int32_t* n_flat;                  // the stream's length
  long long flat_cap;               // entries the stream holds (more: MD_EOVERFLOW)
  int32_t* work;                    // next chunk of the pair kernel
  unsigned int* work_done;          // blocks of the pair kernel that finished
  // FP64 half-list path
  uint32_t* fwd;                    // [molecule * cap_v + front slot]: pairbuf entry of the pair
  dvec4 *pairbuf, *fpart;           // pairbuf [molecule * cap_v + back slot] (+1 spare)
  // wall and cells
  dvec4* wpos;
  float4* wlpos;
  float4* wlpos_lo;                 // and the wall's
  int32_t* wstart;                  // n_cells + 1
  int32_t *vcount, *vstart;         // n_cells, n_cells + 1
  int32_t* scan_tiles;              // tile sums of the cell scan
  const int32_t* cell_rep;          // replica of each cell
  float4* xf;                       // absolute FP32 positions (small-system kernel; else NULL)
  float4* xf_alt;                   // and their second buffer (positions: pos_alt)
  const float4* wxf;                // and the wall's (static)
  const int32_t* row_cell;          // first cell of each row of cells (fixed iy, iz of a replica)
  const int32_t* wnear;             // wall atoms in each cell's 27-cell neighbourhood
  const RepDev* reps;
  const double* cell_ctr;           // per replica: ncx x-centres, ncy y-centres, ncz z-centres
  const PoreDev* pores;
  // per-replica / global scalars
  double* lambda;                   // per replica
  int32_t* any_scale;
  long long* step;
  int32_t* force_rebuild;           // set by the host or by a molecule past skin/2; cleared by the
                                    // pair kernel
  unsigned long long* rep_disp2;    // per replica: the largest squared displacement since its
                                    // last build among molecules past the grouping threshold (bit
                                    // pattern of a double; 0 below it); all-ones bytes when the
                                    // host asks for a rebuild; cleared by the pair kernel
  int32_t* act_cells;               // cells with molecules of the replicas being rebuilt
  int32_t* act_rep;                 // and their replicas
  int32_t* act_home;                // and their coordinates (ix | iy << 10 | iz << 20)
  int32_t* n_act;                   // their number
  int32_t* kick_pending;            // 1: the second half-kick of the last step is still owed (the
                                    // FP64 atomic form defers it into the next first half-kick)
  long long* thermo_owed;           // the step whose Berendsen scaling is still owed (0: none):
                                    // paid by the next step kernel, or by launch_settle
  unsigned long long* bar_arrive;   // the step kernels' grid barrier: arrivals at the current one
  unsigned long long* bar_release;  // and its generation (advanced by each completed barrier)
  unsigned int* kick_done;          // last-block detection in k_kick_pending
  unsigned int* chain_done;         // last-block detection in k_list_build
  int32_t* status;                  // [0] sticky status bits; [1] the source line of the first
                                    // failed index check (checked build)
  unsigned int* blk_done;           // last-block detection in k_integrate_first
  unsigned long long* n_rebuilds;
  unsigned long long* pair_count;   // 2 x pairs within cutoff, summed over steps (whole context)
  unsigned long long* launch_count; // kernels launched by the library
  int32_t* max_nb;
  // observables (per molecule, then per replica)
  double *pe_i, *pevw_i, *vir_i, *virw_i, *d2w_i;
  int32_t *cnt_vv_i, *cnt_vw_i;
  unsigned long long *occ, *ads, *prof;  // per pore, per group, per group*bin
  double* rep_part;                 // per (replica, chunk) partial sums, 8 each
  double* rep_sums;                 // per replica: ke, pe_vv, pe_vw, vir_vv, vir_vw, pairs_vv,
                                    // pairs_vw
  double *pore_part, *pore_press;   // per (replica, chunk, pore) partials; per pore pressure
  int32_t max_pores;                // most pores of any replica (>= 1)
  int32_t n_total, n_wall_total, n_cells, n_reps;
  int32_t n_rows;                   // rows of cells over every replica
  int32_t rep_chunks;               // partial-sum chunks per replica
};

struct Tuning {
  int force_block = 256;
  int force_blocks_per_sm_fp64 = 1;   // resident blocks per SM of the pair kernels (grid size)
  int force_blocks_per_sm_mixed = 4;
  int tpp_fp64 = 2;                   // lanes sharing one molecule's list in the pair kernels;
                                      // 32: the FP64 packed kernel (lanes share packed pairs);
                                      // 64 (kFlatTpp): the flat stream (atomic form)
  int tpp_mixed = 4;
  int gather_tpp = 2;                 // lanes per molecule in the FP64 reverse gather
  int lpt = 1;                        // process molecules longest list first
  int atomic_acc = 0;                 // FP64: reaction forces by atomic adds (no gather)
  int all_pairs = 0;                  // FP64: every pair each step, no lists (the paper's F1)
  int cells = 0;                      // cell-tiled pair kernel: no Verlet lists (pair_method 3)
  int small = 0;                      // whole steps in one persistent launch (pair_method 4)
  int static_chunks = 0;              // atomic list kernels: static round-robin chunk walk
  int list_mode = 0;                  // list build: 0 the device chooses by occupancy, 1 a warp
                                      // per cell, 2 a thread per molecule
  int flat_fill = 0;                  // rebuilds fill the flat stream and the processing order
                                      // whatever the kernel (the tuner's timings)
  int small_blocks_per_sm = 1;        // blocks of the small-system kernel an SM holds at once
  int df64 = 0;                       // FP64 context, pair terms in double-float (FP32 pairs)
  int sm_count = 152;
  int integrate_blocks_per_sm = 1;    // blocks of the step kernel an SM holds at once
};

// carve predicate of a pore at offset (dx, dy) from its axis and height z (slab half-thickness h)
// floor of a prism pore: z = h - depth for a blind pore (0 < depth < 2h), else below the slab
__host__ __device__ inline double prism_floor(double depth, double h) {
  return (depth > 0.0 && depth < 2.0 * h) ? h - depth : -2.0 * h;
}

__host__ __device__ inline bool in_pore(int kind, double r0, double r1, double rcav, double width,
                                        double dx, double dy, double z, double h) {
  double rxy2 = dx * dx + dy * dy;
  switch (kind) {
    case 1: return rxy2 < r0 * r0;
    case 2: return sqrt(rxy2) < r0 + (r1 - r0) * (z + h) / (2.0 * h);
    case 3: return fabs(dy) < 0.5 * width;
    case 4: return rxy2 < r0 * r0 || rxy2 + z * z < rcav * rcav;
    case 5: return fabs(dx) < r0 && fabs(dy) < r1 && z > prism_floor(width, h);
    default: return false;
  }
}

__host__ __device__ inline int cell_coord(double u, double half, double l, int nc) {
  int c = (int)floor((u + half) / l);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// the same with the inverse side (a multiplication: FP64 division is a long sequence on this part)
__host__ __device__ inline int cell_coord_mul(double u, double half, double il, int nc) {
  int c = (int)floor((u + half) * il);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Conditional-node handles of one captured step (unused when launched outside a graph).
struct StepConds {
  cudaGraphConditionalHandle rebuild = 0;
  int use = 0;
  int has_rebuild = 1;              // 0: no rebuild node (all-pairs mode)
};

// ---- launchers (md_kernels.cu); all enqueue on `s` and never synchronise
// flags of the first half-kick: clear the forces (the atomic pair pass adds into them); refresh
// the FP32 cell-local offsets (read by the mixed pair kernel and the packed FP64 kernel's screen)
constexpr int kIntZeroForces = 1;
constexpr int kIntLocalOffsets = 2;
constexpr int kIntLocalOffsetsLo = 4;  // also their double-float remainders
void launch_integrate_first(const Arrays& a, const PotDev& p, bool mixed, const StepConds& c,
                            int flags, const Tuning& t, cudaStream_t s);
void launch_rebuild(const Arrays& a, const PotDev& p, const Tuning& t, bool mixed, cudaStream_t s);
// pair forces at the current positions; with `kick` the FP64 reverse gather is fused with the
// second half-kick (Fig. 3), otherwise the gather only writes the forces
cudaError_t configure_kernels(int* integrate_per_sm, int* small_per_sm);
// small systems (pair_method 4): n whole MD steps in one cooperative launch (n = 0: the forces at
// the current positions only)
constexpr int kSmallMax = 16384;      // molecules of a context the small-system method takes
void launch_small_steps(const Arrays& a, const PotDev& p, const Tuning& t, int nsteps,
                        cudaStream_t s);
// state transfer through device staging rows (caller order, xyz interleaved). The load checks
// the rows first (positions inside the box, planar replicas in the plane) and loads nothing if
// any fails; *bad (kNoBadRow beforehand) receives the lowest failing row k as 3 k (outside the
// box), 3 k + 1 (off the plane) or 3 k + 2 (a non-finite velocity). keep_order (the list methods):
// the records keep their stored order and raise the rebuild flags by the skin test (which must be
// clear beforehand); otherwise the stored order restarts as the caller's and a full rebuild must
// follow.
constexpr int kNoBadRow = 0x7f7f7f7f;  // the byte pattern 0x7f repeated (a memset)
void launch_load_state(const Arrays& a, const PotDev& p, const double* xin, const double* vin,
                       int off, int n, int* bad, bool keep_order, cudaStream_t s);
void launch_store_rows(const Arrays& a, const dvec4* src, double* out, int off, int n,
                       cudaStream_t s);
// the pair kernel alone (no clearing, gather or kick): for timing the dominant kernel
void launch_pair_pass(const Arrays& a, const PotDev& p, bool mixed, const Tuning& t,
                      cudaStream_t s);
void launch_forces(const Arrays& a, const PotDev& p, bool mixed, bool stats, bool kick,
                   const Tuning& t, cudaStream_t s);
// pay what the last step left owed -- its deferred second half-kick and its Berendsen scaling --
// before anything outside a step reads or replaces velocities
void launch_settle(const Arrays& a, const PotDev& p, cudaStream_t s);
// a check of the bounded grid-barrier wait: raises the timeout status on purpose (about a second)
void launch_barrier_check(const Arrays& a, const PotDev& p, cudaStream_t s);
void launch_observables(const Arrays& a, const PotDev& p, cudaStream_t s);

}  // namespace mdk
