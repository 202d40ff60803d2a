/*
 * md.h -- C ABI of the GB300 (sm_103a) molecular-dynamics library for water vapour near atomistic
 * pore walls (Korenkov, Nikonov, Popovicova, arXiv:1812.07993).
 *
 * What one MD step computes (per replica, reduced Lennard-Jones units, sigma = eps = m = k_B = 1):
 *   1. first half-kick and drift (Sec. 2 velocity Verlet; Fig. 2):
 *        v <- v + (dt/2) f/m ;  r <- r + dt v
 *      then specular reflection at z = +-Lz/2, off the solid for hard walls (md_wall_model),
 *      and periodic wrap of x, y into [-L/2, L/2);
 *   2. neighbour-list maintenance: when any molecule has moved more than skin/2 since the last
 *      build, particles are binned into cells (counting sort) and Verlet lists rebuilt;
 *   3. forces at r(t+dt) (Sec. 2, Eq. 2; Fig. 1): f_i = -dU/dr_i with U the Lennard-Jones 12-6
 *      potential (Sec. 2) truncated at rc (vapour-vapour: eps, sigma, rc; vapour-wall: eps_w,
 *      sigma_w, rc_w; wall atoms are fixed and feel no force);
 *   4. second half-kick (Fig. 3): v <- v + (dt/2) f/m;
 *   5. Berendsen scaling (Sec. 2; Fig. 4) when the step counter reaches a multiple of
 *      thermostat_every: v <- lambda v, lambda = sqrt(1 + (n_th dt / tau_B)(T0/T - 1)),
 *      T = m sum v^2 / (d N), d = 3 (or 2 for a planar system).
 * Observables (on demand): kinetic / potential energy, the pair virial sum_{pairs} r_ij . F_ij
 * (the sum in the virial pressure of Sec. 2), pairs within the cutoff, pore occupancy, adsorbed
 * count and axial density profile per pore.
 *
 * Conventions
 *   - Box centred at the origin: x in [-Lx/2, Lx/2), y in [-Ly/2, Ly/2) periodic; z in
 *     [-Lz/2, Lz/2] with reflecting ends. Positions/velocities/forces are FP64, xyz interleaved
 *     (3*n doubles), in the caller's molecule order.
 *   - Every pointer argument named host_* or documented as "host" is host memory owned by the
 *     caller; the library copies from/to it and keeps no reference after the call returns.
 *     The library owns all device memory it allocates and frees it in md_destroy.
 *   - Work is enqueued on the CUDA stream given at creation (NULL: the library creates a
 *     non-blocking stream of its own and destroys it in md_destroy).
 *     md_step is asynchronous; md_sync, md_get_* and md_observables synchronise that stream.
 *   - Errors: every entry point returns an md_status; no exception or abort crosses the ABI.
 *     Conditions found on the device (list overflow, unstable motion, a spin wait that ran out)
 *     are sticky per context: once set, later steps do no work and every call returns the code.
 *     md_last_error gives a one-line description.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef MD_H
#define MD_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_API_VERSION 1

typedef enum {
  MD_OK = 0,
  MD_EINVAL = 1,     /* invalid argument (message in md_last_error) */
  MD_ENOMEM = 2,     /* a device or host allocation failed */
  MD_ECUDA = 3,      /* a CUDA runtime call failed */
  MD_EOVERFLOW = 4,  /* a neighbour list or cell exceeded its capacity */
  MD_EUNSTABLE = 5,  /* a molecule left the box after reflection and wrap, or its position became
                        non-finite (a molecule that moves more than skin/2 between list builds
                        is not an error: the lists are rebuilt within the same step) */
  MD_ETIMEOUT = 6,   /* a bounded device spin wait gave up */
  MD_EBOUNDS = 7     /* the checked build (compiled with -DMD_CHECKED, libmd_checked.so) found an
                        index read from device data -- a list entry, the processing order, a pair
                        slot, a cell or sort index -- outside its array; the access was replaced by
                        an in-bounds one and the status made sticky. The normal build never
                        returns it. */
} md_status;

/* MD_PREC_DF64: an FP64 context (positions, integration, cutoff decisions, accumulation, observables)
 * whose pair terms run in double-float arithmetic -- each value a pair of FP32 numbers hi + lo,
 * combined by error-free transformations (Dekker; Knuth; Joldes, Muller and Popescu 2017) -- on
 * FP32 cell-local offsets split the same way: ~2^-44 relative per pair term, against 2^-53 for
 * FP64, with the work on the FP32 pipe. force_accumulate 2 (the default here): half list with FP64
 * atomic reaction forces; 1: full list, each pair from both ends, no atomics, bit-for-bit
 * reproducible. No force_tpp 32 and no all-pairs method. */
typedef enum { MD_PREC_FP64 = 0, MD_PREC_MIXED = 1, MD_PREC_DF64 = 2 } md_precision;

typedef enum {
  MD_PORE_CYLINDER = 1,   /* dx^2 + dy^2 < r0^2 */
  MD_PORE_CONE = 2,       /* sqrt(dx^2 + dy^2) < r0 + (r1 - r0)(z + h)/(2h), narrow end at z = -h */
  MD_PORE_SLIT = 3,       /* |dy| < width/2, spanning the whole x extent */
  MD_PORE_INKBOTTLE = 4,  /* dx^2 + dy^2 < r0^2  or  dx^2 + dy^2 + z^2 < r_cavity^2 */
  MD_PORE_PRISM = 5       /* |dx| < r0 and |dy| < r1 and z > h - width: a rectangular pore open at
                             the slab's top face z = +h with a floor at z = h - width when
                             0 < width < 2h (otherwise through the slab) -- the paper's pore shape
                             (Sec. 4 and Sec. 5) */
} md_pore_kind;

typedef enum {
  MD_WALL_ATOMS = 0,      /* fixed Lennard-Jones wall atoms (the default) */
  MD_WALL_HARD = 1        /* no wall atoms: the slab |z| < h minus the pores is a solid that
                             reflects molecules specularly (the paper's reflecting pore walls,
                             Sec. 4). A molecule that ends a drift inside the solid is mirrored in
                             the face it crossed: the slab face on its side if it came from outside
                             the slab, else the side walls (prism |dx| = r0, |dy| = r1; slit
                             |dy| = width/2) and the floor of the pore it came from. Pores must be
                             prisms or slits (axis-aligned faces). */
} md_wall_model;

/* One pore carved through the wall slab |z| < h. (dx, dy) is the minimum-image offset of a point
 * from the pore axis (cx, cy). The carve predicates above decide which wall sites are removed
 * when the library generates the wall, and which molecules count toward the pore's occupancy. */
typedef struct {
  int32_t kind;            /* md_pore_kind */
  double cx, cy;           /* axis position */
  double r0, r1;           /* radius (cylinder, neck), cone radii at z = -h and z = +h;
                              prism half-sides in x and y */
  double r_cavity;         /* ink-bottle cavity radius */
  double width;            /* slit width; prism depth from the top face */
} md_pore;

/* One independent system (replica). */
typedef struct {
  double Lx, Ly, Lz;       /* box */
  int64_t n_vapor;         /* mobile molecules */
  const double* x0;        /* host, 3*n_vapor initial positions (inside the box) */
  const double* v0;        /* host, 3*n_vapor initial velocities */
  double T0;               /* thermostat target temperature */
  double dt;               /* time step */
  double tau_B;            /* Berendsen rise time; <= 0 means thermostat_every*dt (plain rescale) */
  int32_t thermostat_every;/* n_th; 0 disables the thermostat */
  double slab_half;        /* wall slab |z| < slab_half */
  double lattice_a;        /* simple-cubic wall spacing when the library generates the wall */
  const double* wall_xyz;  /* host, 3*n_wall fixed wall atoms, or NULL: generate the SC lattice
                              -L/2 + (i + 1/2) a on each axis, |z| < slab_half, minus the pores */
  int64_t n_wall;          /* length of wall_xyz (ignored when wall_xyz is NULL) */
  const md_pore* pores;    /* host, n_pores pores (may be NULL when n_pores == 0) */
  int32_t n_pores;
  int32_t dims;            /* 0 or 3: three-dimensional; 2: planar system in the x-z plane (every
                              molecule at y = 0 with vy = 0; needs wall_model MD_WALL_HARD and
                              prism pores), temperature T = m sum v^2 / (2N) -- the paper's 2D
                              simulation (Sec. 4) */
  int32_t wall_model;      /* md_wall_model */
} md_system;

/* Interaction, list and observable parameters shared by every replica of a context. */
typedef struct {
  double eps, sigma, mass, rc;        /* vapour-vapour Lennard-Jones (cut at rc, strict r < rc) */
  double eps_w, sigma_w, rc_w;        /* vapour-wall Lennard-Jones */
  double skin;                        /* Verlet skin: lists hold pairs with
                                         r < max(rc, rc_w) + skin */
  int32_t shift_energy;               /* 1: energy per pair is U(r) - U(cutoff) */
  int32_t precision;                  /* md_precision: FP64 pair terms, FP32 pair terms with
                                         compensated accumulation and FP64 integration, or
                                         double-float pair terms in an FP64 context */
  double r_ads;                       /* adsorbed: nearest wall atom closer than r_ads (<= rc_w) */
  double bin_width;                   /* axial density-profile bin width */
  int32_t max_neighbors;              /* vapour neighbours a molecule may hold (0 = default 160) */
  int32_t max_wall_neighbors;         /* wall neighbours a molecule may hold (0 = default 224);
                                         one list holds both, of max_neighbors +
                                         max_wall_neighbors entries (at most 1023) */
  double cell_size;                   /* minimum side of the cells (0: the list radius
                                         max(rc, rc_w) + skin, the smallest that works); larger
                                         cells hold more molecules each, which changes only the
                                         speed of the cell sort and the list build: the autotuner
                                         chooses it per size class */
} md_potential;

/* Launch-shape knobs (0 in a field = keep the current value). */
typedef struct {
  int32_t force_block;     /* threads per block of the pair-force kernel: 128 or 256 */
  int32_t force_blocks_per_sm; /* resident pair-kernel blocks per SM: the grid is SMs x this and
                              warps fetch chunks of molecules dynamically (1..32) */
  int32_t force_tpp;       /* lanes that split one molecule's neighbour list: 1, 2, 4, 8 or 16;
                              FP64 also 32: a warp owns 32 molecules, screens their lists in
                              FP32 and packs the surviving pairs so that every lane of the
                              FP64 pair terms is busy; 64 (force_accumulate 2 only, every
                              precision): the flat stream -- at each rebuild the front rows of
                              all molecules are copied into one stream of entries (allocated on
                              first use: up to 128 entries a molecule on average, more is
                              MD_EOVERFLOW), which the warps split evenly, 32 entries at a time;
                              each entry is screened in FP32 and (FP64, double-float) the
                              survivors are queued in registers and evaluated 32 at a time; both
                              ends of a pair receive its force by FP64 atomic adds (for dilute
                              systems: a few entries per row). order_by_length and chunk_walk do
                              not apply to it */
  int32_t order_by_length; /* 1: process molecules longest list first; 2: in cell order */
  int32_t use_graph;       /* 1: md_step replays a captured CUDA graph; 2: plain launches */
  int32_t steps_per_graph; /* MD steps captured per graph replay */
  int32_t force_accumulate; /* 1: deterministic (bit-for-bit reproducible) -- FP64: each vapour
                              pair's force is stored in the partner's slot and every molecule sums
                              its slots in list order; mixed: every molecule sums its whole row.
                              2: each vapour pair is evaluated once and its reaction goes to the
                              partner by an FP64 atomic add (no gather; the second half-kick of a
                              step is deferred into the next step's first); the summation order
                              varies from run to run, so results agree with mode 1 to rounding
                              only. Changing it rebuilds the lists (synchronises). */
  int32_t pair_method;     /* 1: Verlet lists (default); 2 (FP64 only): every pair every step, one
                              thread per molecule summing over all molecules and wall atoms of
                              its replica (the paper's F1 form, Sec. 3, Fig. 1; O(N^2), for small
                              systems), no list rebuilds while on; 3: no Verlet lists -- a warp
                              stages the FP32 offsets of a chunk's 27 neighbour cells in shared
                              memory, screens every staged candidate, queues the pairs that may lie
                              within the cutoff and evaluates them with every lane busy, reaction
                              forces by FP64 atomic adds (force_accumulate 2 only); the rebuild is
                              then the cell sort alone; 4 (FP64, at most 16384 molecules): small
                              systems -- md_step(n) runs whole steps in cooperative launches (up to
                              1000 steps each) with no lists and no sorting: per step every
                              molecule advances, a bounded grid barrier, then a warp per molecule
                              screens every vapour molecule of its replica and the wall atoms of
                              its 27 cells in FP32 and evaluates the candidates in FP64, summing in
                              a fixed order (bit-for-bit reproducible), with the second half-kick;
                              the paper's system sizes (Sec. 4, Sec. 5). Same pair set and forces in
                              every method. */
  int32_t chunk_walk;      /* the atomic Verlet-list kernels (force_accumulate 2, force_tpp 1 to
                              16): 1 dynamic -- every warp takes its next chunk of molecules from a
                              work counter; 2 static -- warp w takes chunks w, w + W, ... of the
                              length-ordered molecules, with the next chunk's molecule index loaded
                              while this chunk runs (two round trips to memory fewer per chunk) */
  int32_t list_build;      /* the Verlet-list build: 1 (default) the device chooses at each rebuild
                              -- a thread per molecule when the rebuilding replicas hold at least
                              65,536 molecules at under 2.5 per occupied cell (dilute vapour), else
                              a warp per cell;
                              2 a warp per cell; 3 a thread per molecule. Both give the same lists,
                              entry for entry. */
} md_tuning;

typedef struct {
  int64_t step;            /* completed MD steps */
  int64_t n_vapor, n_wall;
  double ke, pe, pe_vv, pe_vw;
  double T;                /* m sum v^2 / (3 N) */
  double virial_vv, virial_vw;   /* sum over pairs within cutoff of r_ij . F_ij */
  int64_t pairs_vv, pairs_vw;    /* unique pairs within cutoff at the current positions */
  int64_t occupancy;       /* sum over pores */
  int64_t adsorbed;        /* sum over groups */
  int32_t n_groups;        /* max(n_pores, 1) */
  int32_t n_bins;          /* ceil(Lz / bin_width) */
  int64_t n_rebuilds;      /* neighbour-list builds since creation (whole context) */
  int64_t pair_evals_total;/* pairs within cutoff summed over every step run so far
                              (whole context: unique vapour-vapour + vapour-wall) */
  int32_t max_list_used;   /* longest neighbour list of any build so far (whole context); with
                              force_accumulate 2 the rows hold half lists (partners j > i and
                              wall atoms) */
  int32_t list_capacity;   /* max_neighbors + max_wall_neighbors */
} md_obs;

typedef struct md_ctx md_ctx; /* opaque, library-owned */

/* Create a context holding one replica on the current CUDA device: the system of Sec. 2 (vapour
 * molecules under the Lennard-Jones potential, Eq. 2) around the pore walls of Sec. 4 (2D) and
 * Sec. 5 (3D).
 * stream: a cudaStream_t on which all work is enqueued (NULL: a library-owned stream).
 * On failure *out is NULL and md_last_error(NULL) describes the failure (per host thread).
 * Copies every host input. Builds (or takes) the wall, bins it once, builds the first lists and
 * evaluates the initial forces. Returns MD_EINVAL for inconsistent parameters (cutoff + skin not
 * below half the periodic box, non-positive sizes, non-finite parameters, molecules outside the
 * box, r_ads > rc_w). */
md_status md_create(const md_system* sys, const md_potential* pot, void* stream, md_ctx** out);

/* Create a context holding n_replicas independent systems that advance together: every kernel
 * launch covers all replicas (uneven sizes allowed). Same rules as md_create per replica. Each
 * replica is a system of Sec. 2; batching them is not in the paper. */
md_status md_create_batch(const md_system* systems, int32_t n_replicas, const md_potential* pot,
                          void* stream, md_ctx** out);

/* Replace the launch-shape knobs; takes effect at the next launch. Changing order_by_length
 * rebuilds the lists (synchronises). The paper picks its threads per block by hand (Sec. 4 and
 * Sec. 5); these knobs and md_get_tuning have no other counterpart there. */
md_status md_set_tuning(md_ctx* ctx, const md_tuning* t);
md_status md_get_tuning(const md_ctx* ctx, md_tuning* t);

/* Autotuner (the paper scans threads per block by hand, Sec. 4 and Sec. 5, Figs. 7 and 12): time
 * the pair-force evaluation (md_compute_forces) for every launch shape of a fixed candidate set --
 * force_tpp {1,2,4,8,16, 32 at FP64, and 64 in the atomic form} x force_blocks_per_sm {1,2,4,8} x
 * force_block {128,256} x order_by_length {on,off} on the Verlet lists (in the atomic form also x
 * chunk_walk {dynamic, static} at force_tpp 1 to 16), and, in the atomic form
 * (force_accumulate 2),
 * the cell method (pair_method 3) x force_blocks_per_sm {1,2,4} x force_block {128,256}. Once the
 * caller has set pair_method with md_set_tuning, the tuner keeps that method and times its shapes
 * alone -- with
 * CUDA events on the context's stream (median of `trials` launches each, trials clamped to
 * [3, 101]), then apply the fastest. Positions and velocities are unchanged; forces are recomputed
 * at the same positions. *best and *best_us (either may be NULL) receive the chosen shape and its
 * median time in microseconds. Synchronises. */
md_status md_autotune(md_ctx* ctx, int32_t trials, md_tuning* best, double* best_us);

/* Enqueue n velocity-Verlet steps (Sec. 2; Figs. 1-4: steps 1-5 above) for every replica
 * (asynchronous). Returns a sticky device status found by earlier work, if any, without waiting
 * for the GPU. */
md_status md_step(md_ctx* ctx, int64_t n);

/* Wait for all enqueued work; returns the sticky device status (no counterpart in the paper). */
md_status md_sync(md_ctx* ctx);

/* Copy replica state -- the positions and velocities of Sec. 2, Eq. 1 -- to caller-owned host
 * arrays (3*n_vapor each, caller's molecule order).
 * replica = -1 copies every replica, concatenated in replica order (3 * total vapour each).
 * x: positions wrapped into the box; v: velocities; either may be NULL. The rows are put into
 * caller order on the device and copied with one cudaMemcpyAsync per array (pinned host memory
 * makes it a DMA at full link speed). Synchronises. */
md_status md_get_state(md_ctx* ctx, int32_t replica, double* x, double* v);

/* Overwrite replica state -- the positions and velocities of Sec. 2, Eq. 1 -- from host arrays
 * (3*n_vapor each, caller's order). Positions must lie inside the box (x, y in [-L/2, L/2), z in
 * [-Lz/2, Lz/2]; a planar replica's y and vy must be 0) and velocities must be finite.
 * replica = -1 sets every replica from arrays concatenated in replica order.
 * - The rows go by one copy per array into device staging rows.
 * - A kernel checks every row there, then a kernel writes the records only if all rows passed.
 * - The list methods keep the stored order: each record takes its own molecule's row, and lists
 *   are rebuilt only for the replicas where some molecule lies at least skin/2 from its position
 *   at the last build (a step's skin test, item 2 at the top of this header). The all-pairs and
 *   small-system methods keep no lists. Forces are re-evaluated.
 * A failing row gives MD_EINVAL, with its replica and molecule in md_last_error, and leaves the
 * positions and velocities as they were (an owed half-kick is still paid). The step counter is
 * unchanged. Synchronises once at the start and once at the end. */
md_status md_set_state(md_ctx* ctx, int32_t replica, const double* x, const double* v);

/* Enqueue one evaluation of the forces at the current positions with the same pair-force kernel
 * and launch shape the step uses (Eq. 2, Fig. 1), without moving molecules or rebuilding lists.
 * Asynchronous; meant for timing the pair kernel in isolation. */
md_status md_compute_forces(md_ctx* ctx);

/* Enqueue the pair kernel alone (F1: Fig. 1, Eq. 2) -- the dominant kernel of the step (the FP64
 * half-list or atomic pass, the all-pairs pass, or the mixed-precision pass) -- with no clearing,
 * gather or kick, so that its duration can be timed with events on the context's stream. It leaves the forces
 * incomplete (or, in the atomic form, added twice): call md_compute_forces afterwards before
 * reading forces or stepping. Asynchronous. */
md_status md_pair_pass(md_ctx* ctx);

/* Enqueue the rebuild chain alone for every replica, at the current positions. The chain is not
 * in the paper, whose F1 sums over all particles (Fig. 1, Sec. 3): its cell and Verlet lists
 * replace that sum. The chain is the counting sort of the vapour by cell, the Verlet lists with
 * skin and the processing order (the FP64 deterministic form also rebuilds its pair map; the cell
 * method, pair_method 3, has the counting sort alone). No forces are evaluated, and none change: the
 * molecules' records, forces included, move to their new sorted places together, and every
 * read-back is in caller order as before. Meant for timing the chain with events on the
 * context's stream; md_step continues from it as from any rebuild, and n_rebuilds counts it.
 * Asynchronous. MD_EINVAL in the all-pairs mode (pair_method 2), which keeps no lists; a list
 * overflow found by the chain is reported by the next synchronising call, as in md_step. */
md_status md_rebuild_lists(md_ctx* ctx);

/* Host<->device bytes the library has copied for this context since creation (state uploads,
 * read-backs, status words). Either pointer may be NULL. No counterpart in the paper. */
md_status md_transfer_bytes(const md_ctx* ctx, int64_t* h2d, int64_t* d2h);

/* Copy the forces of the last evaluation (Eq. 2, Fig. 1; at the current positions) to host f
 * (3*n_vapor; with replica = -1, every replica concatenated in replica order). Synchronises. */
md_status md_get_forces(md_ctx* ctx, int32_t replica, double* f);

/* Observables of one replica at the current state. Fills *out; when non-NULL the arrays receive
 * occupancy[n_pores], adsorbed[n_groups], profile[n_groups * n_bins] (group-major) and
 * pore_pressure[n_pores]. A molecule belongs to the pore whose axis is nearest in xy (slits:
 * |dy|); ties go to the lower pore index. bins: floor((z + Lz/2)/bin_width), the last bin closed.
 * pore_pressure: the virial pressure of Sec. 2 in each pore,
 *   P = (sum_i m v_i^2 + sum_i W_i) / (3 V),
 * over the molecules inside the pore (the occupancy predicate), W_i = half of r_ij . F_ij of each
 * vapour pair plus r_iw . F_iw of each wall pair of molecule i, V the volume of the pore's carved
 * region inside the slab. The forces of the last step are not changed. Synchronises. */
md_status md_observables(md_ctx* ctx, int32_t replica, md_obs* out, int64_t* occupancy,
                         int64_t* adsorbed, int64_t* profile, double* pore_pressure);

/* FP64 forces that allocate no memory (the paper has no counterpart: it is a service for callers
 * that cannot allocate device memory, such as an application whose own pool allocator already
 * holds nearly all of it, so a cudaMalloc would fail, or a latency-critical host thread that must
 * not meet the implicit device synchronisation of cudaFree).
 * Computes f_i = sum of Lennard-Jones pair forces (same potential and cutoffs as the context path,
 * eps/sigma/rc and eps_w/sigma_w/rc_w of *pot, FP64) on n_vapor molecules at d_x from each other
 * and from n_wall fixed wall atoms at d_wall, in a box Lx x Ly x Lz centred at the origin
 * (periodic x, y). d_x (3*n_vapor), d_wall (3*n_wall) and d_f (3*n_vapor) are caller-owned DEVICE
 * arrays, xyz interleaved. z must lie in [-Lz/2, Lz/2] (a z outside is binned into the nearest
 * edge cell); x and y outside [-L/2, L/2) are wrapped periodically before binning and in the
 * distances. Work is enqueued on `stream` (NULL = legacy default stream) and is asynchronous.
 * Non-finite box sides or potential parameters give MD_EINVAL. A CUDA error already pending on
 * the calling thread (from the caller's own earlier work) makes the call return MD_ECUDA before
 * any launch, and is left set for the caller.
 * Scratch: a fixed array of about 4 MB inside the library, reserved on every GPU that loads the
 * library until the process exits. Limits: n_vapor + n_wall <= 262144 atoms and at most 65536
 * cells of side >= max(rc, rc_w), with at least 3 cells across x and y; larger inputs return
 * MD_EINVAL with the reason in err (err_len bytes, may be NULL). The first call on a device looks
 * up the scratch address once (cudaGetSymbolAddress, with that device current): make that first
 * call before any stream capture. All calls share the scratch and its contents persist between
 * calls: calls whose GPU work overlaps (other streams, other host threads) race and must not. */
md_status md_forces_noalloc(const md_potential* pot, double Lx, double Ly, double Lz,
                            const double* d_x, int64_t n_vapor, const double* d_wall,
                            int64_t n_wall, double* d_f, void* stream, char* err, int32_t err_len);

/* Copy the wall atoms of a replica (3*n_wall doubles, as generated or given): the fixed atoms of
 * the pore walls of Sec. 4 and Sec. 5. */
md_status md_get_wall(md_ctx* ctx, int32_t replica, double* wall_xyz);

/* Sizes of one replica (no counterpart in the paper). */
md_status md_get_sizes(const md_ctx* ctx, int32_t replica, int64_t* n_vapor, int64_t* n_wall,
                       int32_t* n_groups, int32_t* n_bins);

/* Kernels the library has launched since creation, counted on the device (kernels inside a
 * graph's skipped conditional branches do not run and are not counted). Synchronises. No
 * counterpart in the paper. */
int64_t md_kernel_launches(const md_ctx* ctx);

/* Check of the failure path for device waits (the paper has no counterpart). The step kernels meet
 * at a grid barrier (the thermostat's sums, and every step of the small-system method), whose
 * waits are bounded: a block that waits too long raises MD_ETIMEOUT and returns instead of
 * hanging. This call makes that happen on purpose -- a kernel of two blocks in which one never
 * arrives -- waits for the other to give up (about a second), checks that the device reported
 * MD_ETIMEOUT, then clears the status and the barrier so that the context goes on as before.
 * *seconds (may be NULL) receives the GPU time until the wait gave up. Returns MD_OK when the
 * timeout was reported, MD_ECUDA otherwise; a status already raised on the context is returned
 * before anything runs. Synchronises. */
md_status md_check_barrier_timeout(md_ctx* ctx, double* seconds);

/* Human-readable text of a status, and the last error message of a context (never NULL);
 * md_last_error(NULL) gives the last md_create / md_create_batch failure of the calling thread.
 * No counterpart in the paper. */
const char* md_status_string(md_status s);
const char* md_last_error(const md_ctx* ctx);

/* Free every resource of the context (synchronises its stream). NULL is ignored. No counterpart
 * in the paper. */
void md_destroy(md_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
