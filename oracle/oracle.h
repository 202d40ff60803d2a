/*
 * oracle.h -- plain FP64 CPU oracle for the water-vapour / pore molecular dynamics.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline /
 * reference legs may load or call it. The CUDA library shares no code, header, table or helper
 * with this file, and neither side includes the other.
 *
 * What it computes, and from where (Korenkov, Nikonov, Popovicova, arXiv:1812.07993):
 *   - Newton's equations m r'' = f  (Sec. 2, Eq. 1) with f_i = -dU/dr_i  (Sec. 2, Eq. 2),
 *     no external field.
 *   - U: Lennard-Jones 12-6 pair potential (Sec. 2), truncated at a cutoff rc (pairs with
 *     r^2 < rc^2 only), energy optionally shifted so that U(rc) = 0; the force is not shifted.
 *     Vapour-vapour pairs use (eps, sigma, rc); vapour-wall pairs use (eps_w, sigma_w, rc_w).
 *     Wall atoms are fixed: they exert forces on vapour and feel none.
 *   - Velocity Verlet (Sec. 2; Figs. 2 and 3): r(t+dt) = r + v dt + a dt^2/2, v(t+dt/2) = v + a dt/2,
 *     forces at r(t+dt) (Fig. 1), v(t+dt) = v(t+dt/2) + a(t+dt) dt/2.
 *   - Berendsen velocity scaling (Sec. 2; Fig. 4): v <- lambda v every n_th steps with
 *     lambda = sqrt(1 + (n_th dt / tau_B)(T0/T - 1)), T = m sum v^2 / (3 N).
 *   - Boundaries: periodic in x and y (minimum image), specular reflection at z = +-Lz/2.
 *   - Observables: pore occupancy, adsorbed count, axial density profile, pair counts, energies,
 *     virial sum_{pairs} r_ij . F_ij (the sum in the virial pressure of Sec. 2).
 *
 * Precision: IEEE FP64, no fast-math, no FMA contraction. Every reduction runs in a fixed order,
 * so results do not depend on the thread count.
 */
#ifndef MD_ORACLE_H
#define MD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double Lx, Ly, Lz;          /* box: x, y in [-L/2, L/2) periodic; z in [-Lz/2, Lz/2] reflecting */
  double eps, sigma, mass, rc;
  double eps_w, sigma_w, rc_w;
  int32_t shift_energy;       /* 1: subtract U(rc) per pair from the energy */
  int32_t thermostat_every;   /* n_th; 0 disables the thermostat */
  double dt, T0, tau_B;       /* tau_B <= 0 means tau_B = n_th * dt (plain rescaling to T0) */
  double slab_half;           /* wall slab |z| < slab_half (occupancy window) */
  double r_ads;               /* adsorbed when the nearest wall atom is closer than r_ads */
  double bin_width;           /* axial profile bin width */
  int32_t dims;               /* 3, or 2: a planar system in x-z (y = 0, vy = 0), T = m sum v^2 / (2N) */
  int32_t hard_walls;         /* 1: no wall atoms; the slab |z| < slab_half minus the pores is a solid
                                 that reflects molecules specularly (the paper's reflecting pore
                                 walls, Sec. 4 and Sec. 5); needs orc_run_geom */
} orc_params;

typedef struct {
  int32_t kind;               /* 1 cylinder, 2 cone, 3 slit, 4 ink-bottle, 5 rectangular prism */
  double cx, cy, r0, r1, r_cavity, width;
  /* prism: |x - cx| < r0, |y - cy| < r1, open at the slab's top face z = +slab_half and closed by
     a floor at z = slab_half - width when 0 < width < 2 slab_half (otherwise a through-pore) */
} orc_pore;

typedef struct {
  double pe_vv, pe_vw;        /* potential energy of vapour-vapour and vapour-wall pairs */
  double vir_vv, vir_vw;      /* sum over pairs of r_ij . F_ij */
  int64_t pairs_vv, pairs_vw; /* unique pairs with r < cutoff */
} orc_stats;

/* Lennard-Jones 12-6 (Sec. 2): u = 4 eps [(s/r)^12 - (s/r)^6]; f_over_r = F(r)/r with
 * F(r) = -dU/dr, so the force on i from j is f_over_r * (r_i - r_j). */
void orc_lj(double r2, double eps, double sigma, double* f_over_r, double* u);

/* Forces (Eq. 2) on n vapour molecules at x (3n, xyz interleaved) from each other and from nw
 * fixed wall atoms w (3nw). Writes f (3n). If d2wall != NULL it receives, per molecule, the
 * squared distance to the nearest wall atom within rc_w (or +inf). method 0 = all pairs,
 * method 1 = plain cell list rebuilt on every call (falls back to all pairs for boxes with fewer
 * than 3 cells across x or y). nthreads <= 0 uses the OpenMP default. Returns 0, or -1 on bad
 * parameters (cutoff not below half the periodic box). */
int orc_forces(const orc_params* p, int64_t n, const double* x, int64_t nw, const double* w,
               double* f, double* d2wall, orc_stats* st, int method, int nthreads);

/* As orc_forces, and when wvir != NULL also each molecule's virial (n values): half of
 * r_ij . F_ij for every vapour pair plus r_iw . F_iw for every wall pair, so that the molecules'
 * virials add up to the pair virial sum. */
int orc_forces_w(const orc_params* p, int64_t n, const double* x, int64_t nw, const double* w,
                 double* f, double* d2wall, double* wvir, orc_stats* st, int method, int nthreads);

/* Volume of a pore's carved region inside the slab |z| < slab_half: the integral over z of the
 * cross-section area (cylinder pi r0^2, cone pi R(z)^2, slit width * Lx, ink-bottle
 * pi max(r0^2, r_cav^2 - z^2), prism 4 r0 r1 above its floor), by composite Simpson quadrature on
 * 20000 intervals over the z range the pore occupies. For dims == 2 the measure is the area in the
 * x-z plane: the cross-section is the length 2 r0 (prism). */
double orc_pore_volume(const orc_params* p, const orc_pore* q);

/* Virial pressure in each pore (Sec. 2): P_q = (sum m v_i^2 + sum W_i) / (dims V_q) over the
 * molecules inside pore q (the occupancy predicate), W_i from orc_forces_w. */
int orc_pore_pressure(const orc_params* p, const orc_pore* pores, int npores, int64_t n,
                      const double* x, const double* v, const double* wvir, double* pressure);

/* Kinetic energy 1/2 m sum v^2. */
double orc_kinetic(const orc_params* p, int64_t n, const double* v);

/* Run nsteps velocity-Verlet steps (Figs. 1-4) from (x, v, f), where f must hold the forces at x.
 * *step is the step counter (incremented per step; the thermostat acts when it becomes a
 * multiple of n_th). ke_log / pe_log (length nsteps, may be NULL) receive the kinetic energy
 * after the second half-kick (before the thermostat) and the potential energy at r(t+dt).
 * d2wall (n, may be NULL) receives the nearest-wall distances of the last force evaluation. */
int orc_run(const orc_params* p, int64_t n, double* x, double* v, double* f, int64_t nw,
            const double* w, int64_t* step, int64_t nsteps, int method, int nthreads,
            double* ke_log, double* pe_log, double* d2wall, orc_stats* last);

/* As orc_run, with the pore geometry that hard walls need: after the drift and the z reflection at
 * the box, a molecule that ends inside the solid (p->hard_walls) is reflected specularly off the
 * face it crossed -- the slab face z = +-slab_half if it came from outside the slab, else the side
 * walls or the floor of the pore it came from (axis-aligned faces: prism and slit pores) -- and
 * x, y are then wrapped. The thermostat uses T = m sum v^2 / (dims N). */
int orc_run_geom(const orc_params* p, const orc_pore* pores, int npores, int64_t n, double* x,
                 double* v, double* f, int64_t nw, const double* w, int64_t* step, int64_t nsteps,
                 int method, int nthreads, double* ke_log, double* pe_log, double* d2wall,
                 orc_stats* last);

/* 1 if point x (3) lies in the solid of a hard-wall system: |z| < slab_half outside every pore. */
int orc_in_solid(const orc_params* p, const orc_pore* pores, int npores, const double* x);

/* Per-pore observables at positions x with nearest-wall distances d2wall (from orc_forces).
 * Groups: one per pore (a molecule belongs to the pore whose axis is nearest in xy; ties go to
 * the lower index), or a single group when npores == 0.
 *   occupancy[npores]       molecules with |z| < slab_half inside the pore's carved region
 *   adsorbed[ngroups]       molecules with d2wall < r_ads^2
 *   profile[ngroups*nbins]  counts in z bins of width bin_width from -Lz/2 (last bin closed)
 * Returns 0, or -1 if nbins is too small for the box. */
int orc_observables(const orc_params* p, const orc_pore* pores, int npores, int64_t n,
                    const double* x, const double* d2wall, int64_t* occupancy, int64_t* adsorbed,
                    int64_t* profile, int nbins);

/* Number of profile bins for a box: ceil(Lz / bin_width). */
int orc_nbins(const orc_params* p);

#ifdef __cplusplus
}
#endif
#endif
