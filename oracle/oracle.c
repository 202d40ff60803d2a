/*
 * oracle.c -- plain FP64 CPU oracle for the water-vapour / pore MD. TEST INFRASTRUCTURE ONLY:
 * loaded by the tests, the smoke check and the benchmark's CPU legs, never by the CUDA library.
 * See oracle.h for what each function computes and which part of the paper it follows.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Sec. 2: Lennard-Jones 12-6.  U(r) = 4 eps [(s/r)^12 - (s/r)^6],
 * F(r) = -dU/dr = (24 eps / r) [2 (s/r)^12 - (s/r)^6]; returned as F(r)/r. */
void orc_lj(double r2, double eps, double sigma, double* f_over_r, double* u) {
  double sr2 = (sigma * sigma) / r2;
  double sr6 = sr2 * sr2 * sr2;
  double sr12 = sr6 * sr6;
  *u = 4.0 * eps * (sr12 - sr6);
  *f_over_r = 24.0 * eps * (2.0 * sr12 - sr6) / r2;
}

/* periodic minimum image for an offset of two wrapped coordinates (|d| < L) */
static double min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

static double energy_shift(double rc, double eps, double sigma, int shift) {
  double f, u;
  if (!shift) return 0.0;
  orc_lj(rc * rc, eps, sigma, &f, &u);
  return u;
}

/* per-molecule partial results, reduced afterwards in molecule order */
typedef struct {
  double fx, fy, fz, pe_vv, pe_vw, vir_vv, vir_vw, d2w;
  int64_t nvv, nvw;
} acc_t;

int orc_forces_w(const orc_params* p, int64_t n, const double* x, int64_t nw, const double* w,
                 double* f, double* d2wall, double* wvir, orc_stats* st, int method, int nthreads);

static void acc_zero(acc_t* a) {
  memset(a, 0, sizeof(*a));
  a->d2w = INFINITY;
}

/* one pair (i with neighbour at offset d = r_i - r_j) */
static void add_pair(acc_t* a, double dx, double dy, double dz, double rc2, double eps,
                     double sigma, double ushift, int is_wall) {
  double r2 = dx * dx + dy * dy + dz * dz;
  double fr, u;
  if (!(r2 < rc2)) return;
  orc_lj(r2, eps, sigma, &fr, &u);
  a->fx += fr * dx;
  a->fy += fr * dy;
  a->fz += fr * dz;
  if (is_wall) {
    a->pe_vw += u - ushift;
    a->vir_vw += fr * r2;
    a->nvw += 1;
    if (r2 < a->d2w) a->d2w = r2;
  } else {
    /* each vapour-vapour pair is visited from both ends: half of it to each */
    a->pe_vv += 0.5 * (u - ushift);
    a->vir_vv += 0.5 * fr * r2;
    a->nvv += 1;
  }
}

/* ---------------------------------------------------------------- all pairs */
static void forces_allpairs(const orc_params* p, int64_t n, const double* x, int64_t nw,
                            const double* w, acc_t* acc) {
  const double rc2 = p->rc * p->rc, rcw2 = p->rc_w * p->rc_w;
  const double us = energy_shift(p->rc, p->eps, p->sigma, p->shift_energy);
  const double usw = energy_shift(p->rc_w, p->eps_w, p->sigma_w, p->shift_energy);
  int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
  for (i = 0; i < n; ++i) {
    acc_t a;
    acc_zero(&a);
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      add_pair(&a, min_image(xi - x[3 * j], p->Lx), min_image(yi - x[3 * j + 1], p->Ly),
               zi - x[3 * j + 2], rc2, p->eps, p->sigma, us, 0);
    }
    for (int64_t k = 0; k < nw; ++k) {
      add_pair(&a, min_image(xi - w[3 * k], p->Lx), min_image(yi - w[3 * k + 1], p->Ly),
               zi - w[3 * k + 2], rcw2, p->eps_w, p->sigma_w, usw, 1);
    }
    acc[i] = a;
  }
}

/* ---------------------------------------------------------------- plain cell list */
typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  int64_t* start; /* ncell + 1 */
  int64_t* idx;   /* particle indices ordered by cell (stable) */
} cells_t;

static int cell_coord(double u, double half, double l, int nc) {
  int c = (int)floor((u + half) / l);
  if (c < 0) c = 0;
  if (c >= nc) c = nc - 1;
  return c;
}

static void cells_build(cells_t* c, const orc_params* p, double rcut, int64_t n, const double* x) {
  c->nx = (int)floor(p->Lx / rcut);
  c->ny = (int)floor(p->Ly / rcut);
  c->nz = (int)floor(p->Lz / rcut);
  if (c->nz < 1) c->nz = 1;
  c->lx = p->Lx / c->nx;
  c->ly = p->Ly / c->ny;
  c->lz = p->Lz / c->nz;
  int64_t ncell = (int64_t)c->nx * c->ny * c->nz;
  c->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  c->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    int a = cell_coord(x[3 * i], 0.5 * p->Lx, c->lx, c->nx);
    int b = cell_coord(x[3 * i + 1], 0.5 * p->Ly, c->ly, c->ny);
    int d = cell_coord(x[3 * i + 2], 0.5 * p->Lz, c->lz, c->nz);
    cid[i] = ((int64_t)d * c->ny + b) * c->nx + a;
    c->start[cid[i] + 1] += 1;
  }
  for (int64_t k = 0; k < ncell; ++k) c->start[k + 1] += c->start[k];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
  memcpy(fill, c->start, sizeof(int64_t) * (size_t)ncell);
  for (int64_t i = 0; i < n; ++i) c->idx[fill[cid[i]]++] = i;
  free(fill);
  free(cid);
}

static void cells_free(cells_t* c) {
  free(c->start);
  free(c->idx);
}

static void forces_cells(const orc_params* p, int64_t n, const double* x, int64_t nw,
                         const double* w, acc_t* acc) {
  const double rc2 = p->rc * p->rc, rcw2 = p->rc_w * p->rc_w;
  const double us = energy_shift(p->rc, p->eps, p->sigma, p->shift_energy);
  const double usw = energy_shift(p->rc_w, p->eps_w, p->sigma_w, p->shift_energy);
  const double rcut = p->rc > p->rc_w ? p->rc : p->rc_w;
  cells_t cv, cw;
  cells_build(&cv, p, rcut, n, x);
  cells_build(&cw, p, rcut, nw, w);
  int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
  for (i = 0; i < n; ++i) {
    acc_t a;
    acc_zero(&a);
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    int ci = cell_coord(xi, 0.5 * p->Lx, cv.lx, cv.nx);
    int cj = cell_coord(yi, 0.5 * p->Ly, cv.ly, cv.ny);
    int ck = cell_coord(zi, 0.5 * p->Lz, cv.lz, cv.nz);
    for (int dk = -1; dk <= 1; ++dk) {
      int kk = ck + dk;
      if (kk < 0 || kk >= cv.nz) continue;
      for (int dj = -1; dj <= 1; ++dj) {
        int jj = (cj + dj + cv.ny) % cv.ny;
        for (int di = -1; di <= 1; ++di) {
          int ii = (ci + di + cv.nx) % cv.nx;
          int64_t cell = ((int64_t)kk * cv.ny + jj) * cv.nx + ii;
          for (int64_t s = cv.start[cell]; s < cv.start[cell + 1]; ++s) {
            int64_t j = cv.idx[s];
            if (j == i) continue;
            add_pair(&a, min_image(xi - x[3 * j], p->Lx), min_image(yi - x[3 * j + 1], p->Ly),
                     zi - x[3 * j + 2], rc2, p->eps, p->sigma, us, 0);
          }
          for (int64_t s = cw.start[cell]; s < cw.start[cell + 1]; ++s) {
            int64_t k = cw.idx[s];
            add_pair(&a, min_image(xi - w[3 * k], p->Lx), min_image(yi - w[3 * k + 1], p->Ly),
                     zi - w[3 * k + 2], rcw2, p->eps_w, p->sigma_w, usw, 1);
          }
        }
      }
    }
    acc[i] = a;
  }
  cells_free(&cv);
  cells_free(&cw);
}

int orc_forces(const orc_params* p, int64_t n, const double* x, int64_t nw, const double* w,
               double* f, double* d2wall, orc_stats* st, int method, int nthreads) {
  return orc_forces_w(p, n, x, nw, w, f, d2wall, NULL, st, method, nthreads);
}

int orc_forces_w(const orc_params* p, int64_t n, const double* x, int64_t nw, const double* w,
                 double* f, double* d2wall, double* wvir, orc_stats* st, int method, int nthreads) {
  const double rcut = p->rc > p->rc_w ? p->rc : p->rc_w;
  if (!(rcut < 0.5 * p->Lx) || !(rcut < 0.5 * p->Ly)) return -1;
#ifdef _OPENMP
  int saved = omp_get_max_threads();
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  acc_t* acc = (acc_t*)malloc(sizeof(acc_t) * (size_t)(n > 0 ? n : 1));
  int cells_ok = (int)floor(p->Lx / rcut) >= 3 && (int)floor(p->Ly / rcut) >= 3;
  if (method == 1 && cells_ok)
    forces_cells(p, n, x, nw, w, acc);
  else
    forces_allpairs(p, n, x, nw, w, acc);
  orc_stats s;
  memset(&s, 0, sizeof(s));
  for (int64_t i = 0; i < n; ++i) {
    f[3 * i] = acc[i].fx;
    f[3 * i + 1] = acc[i].fy;
    f[3 * i + 2] = acc[i].fz;
    if (d2wall) d2wall[i] = acc[i].d2w;
    if (wvir) wvir[i] = acc[i].vir_vv + acc[i].vir_vw;
    s.pe_vv += acc[i].pe_vv;
    s.pe_vw += acc[i].pe_vw;
    s.vir_vv += acc[i].vir_vv;
    s.vir_vw += acc[i].vir_vw;
    s.pairs_vv += acc[i].nvv;
    s.pairs_vw += acc[i].nvw;
  }
  s.pairs_vv /= 2;
  if (st) *st = s;
  free(acc);
#ifdef _OPENMP
  omp_set_num_threads(saved);
#endif
  return 0;
}

double orc_kinetic(const orc_params* p, int64_t n, const double* v) {
  double s = 0.0;
  for (int64_t i = 0; i < 3 * n; ++i) s += v[i] * v[i];
  return 0.5 * p->mass * s;
}

/* specular reflection at z = +-Lz/2 */
static void reflect_box_z(const orc_params* p, double* r, double* v) {
  const double hz = 0.5 * p->Lz;
  if (r[2] > hz) {
    r[2] = p->Lz - r[2];
    v[2] = -v[2];
  } else if (r[2] < -hz) {
    r[2] = -p->Lz - r[2];
    v[2] = -v[2];
  }
}

/* periodic wrap of x and y into [-L/2, L/2) */
static void wrap_xy(const orc_params* p, double* r) {
  if (r[0] >= 0.5 * p->Lx) r[0] -= p->Lx;
  else if (r[0] < -0.5 * p->Lx) r[0] += p->Lx;
  if (r[1] >= 0.5 * p->Ly) r[1] -= p->Ly;
  else if (r[1] < -0.5 * p->Ly) r[1] += p->Ly;
}

int orc_run(const orc_params* p, int64_t n, double* x, double* v, double* f, int64_t nw,
            const double* w, int64_t* step, int64_t nsteps, int method, int nthreads,
            double* ke_log, double* pe_log, double* d2wall, orc_stats* last) {
  if (p->hard_walls) return -1; /* hard walls need the pore geometry: orc_run_geom */
  return orc_run_geom(p, NULL, 0, n, x, v, f, nw, w, step, nsteps, method, nthreads, ke_log,
                      pe_log, d2wall, last);
}

/* floor of a prism pore: z = h - depth for a blind pore (0 < depth < 2h), else below the slab */
static double prism_floor(const orc_pore* q, double h) {
  return (q->width > 0.0 && q->width < 2.0 * h) ? h - q->width : -2.0 * h;
}

/* carved region of a pore at a point (dx, dy = offset from the axis, z) */
static int in_pore(const orc_pore* q, double dx, double dy, double z, double h) {
  double rxy2 = dx * dx + dy * dy;
  switch (q->kind) {
    case 1: return rxy2 < q->r0 * q->r0;
    case 2: return sqrt(rxy2) < q->r0 + (q->r1 - q->r0) * (z + h) / (2.0 * h);
    case 3: return fabs(dy) < 0.5 * q->width;
    case 4: return rxy2 < q->r0 * q->r0 || rxy2 + z * z < q->r_cavity * q->r_cavity;
    case 5: return fabs(dx) < q->r0 && fabs(dy) < q->r1 && z > prism_floor(q, h);
    default: return 0;
  }
}

int orc_in_solid(const orc_params* p, const orc_pore* pores, int npores, const double* r) {
  const double h = p->slab_half;
  if (!(fabs(r[2]) < h)) return 0;
  for (int q = 0; q < npores; ++q) {
    double dx = min_image(r[0] - pores[q].cx, p->Lx), dy = min_image(r[1] - pores[q].cy, p->Ly);
    if (in_pore(&pores[q], dx, dy, r[2], h)) return 0;
  }
  return 1;
}

/* Hard walls: a molecule that ended the drift inside the solid is reflected off the face it
 * crossed. From outside the slab (|z_old| >= h) that is the slab face on its side; from inside a
 * pore it is each side wall (|dx| >= r0 or |dy| >= r1, slit: |dy| >= width/2) it passed and the
 * floor (z <= floor). Specular: the coordinate is mirrored in the face, that velocity component
 * reversed. */
static void reflect_solid(const orc_params* p, const orc_pore* pores, int npores,
                          const double* r_old, double* r, double* v) {
  const double h = p->slab_half;
  if (!orc_in_solid(p, pores, npores, r)) return;
  if (fabs(r_old[2]) >= h) {
    const double face = r_old[2] > 0.0 ? h : -h;
    r[2] = 2.0 * face - r[2];
    v[2] = -v[2];
    return;
  }
  for (int q = 0; q < npores; ++q) {
    const orc_pore* P = &pores[q];
    double dx0 = min_image(r_old[0] - P->cx, p->Lx), dy0 = min_image(r_old[1] - P->cy, p->Ly);
    if (!in_pore(P, dx0, dy0, r_old[2], h)) continue;
    double dx = min_image(r[0] - P->cx, p->Lx), dy = min_image(r[1] - P->cy, p->Ly);
    if (P->kind == 5) {
      if (dx >= P->r0) { r[0] += 2.0 * (P->r0 - dx); v[0] = -v[0]; }
      else if (dx <= -P->r0) { r[0] += 2.0 * (-P->r0 - dx); v[0] = -v[0]; }
      if (dy >= P->r1) { r[1] += 2.0 * (P->r1 - dy); v[1] = -v[1]; }
      else if (dy <= -P->r1) { r[1] += 2.0 * (-P->r1 - dy); v[1] = -v[1]; }
      const double fl = prism_floor(P, h);
      if (r[2] <= fl) { r[2] = 2.0 * fl - r[2]; v[2] = -v[2]; }
    } else if (P->kind == 3) {
      const double hw = 0.5 * P->width;
      if (dy >= hw) { r[1] += 2.0 * (hw - dy); v[1] = -v[1]; }
      else if (dy <= -hw) { r[1] += 2.0 * (-hw - dy); v[1] = -v[1]; }
    }
    return;
  }
}

int orc_run_geom(const orc_params* p, const orc_pore* pores, int npores, int64_t n, double* x,
                 double* v, double* f, int64_t nw, const double* w, int64_t* step, int64_t nsteps,
                 int method, int nthreads, double* ke_log, double* pe_log, double* d2wall,
                 orc_stats* last) {
  const double dt = p->dt, m = p->mass;
  const double dof = p->dims == 2 ? 2.0 : 3.0;
  for (int64_t s = 0; s < nsteps; ++s) {
    /* Fig. 2: r(t+dt) = r(t) + v(t) dt + a(t) dt^2 / 2 ;  v(t+dt/2) = v(t) + a(t) dt / 2 */
    for (int64_t i = 0; i < n; ++i) {
      double r_old[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
      for (int c = 0; c < 3; ++c) {
        double a = f[3 * i + c] / m;
        x[3 * i + c] = x[3 * i + c] + v[3 * i + c] * dt + 0.5 * a * dt * dt;
        v[3 * i + c] = v[3 * i + c] + 0.5 * a * dt;
      }
      reflect_box_z(p, &x[3 * i], &v[3 * i]);
      if (p->hard_walls) reflect_solid(p, pores, npores, r_old, &x[3 * i], &v[3 * i]);
      wrap_xy(p, &x[3 * i]);
    }
    /* Fig. 1: a(t+dt) from the interaction potential at r(t+dt) */
    orc_stats st;
    if (orc_forces(p, n, x, nw, w, f, d2wall, &st, method, nthreads) != 0) return -1;
    /* Fig. 3: v(t+dt) = v(t+dt/2) + a(t+dt) dt / 2 */
    for (int64_t i = 0; i < 3 * n; ++i) v[i] = v[i] + 0.5 * (f[i] / m) * dt;
    *step += 1;
    double ke = orc_kinetic(p, n, v);
    if (ke_log) ke_log[s] = ke;
    if (pe_log) pe_log[s] = st.pe_vv + st.pe_vw;
    if (last) *last = st;
    /* Fig. 4: Berendsen scaling v <- lambda v on every n_th-th step */
    if (p->thermostat_every > 0 && (*step % p->thermostat_every) == 0 && n > 0) {
      double T = 2.0 * ke / (dof * (double)n);
      double tauB = p->tau_B > 0.0 ? p->tau_B : p->thermostat_every * dt;
      double lambda = 1.0;
      if (T > 0.0) lambda = sqrt(1.0 + (p->thermostat_every * dt / tauB) * (p->T0 / T - 1.0));
      for (int64_t i = 0; i < 3 * n; ++i) v[i] = lambda * v[i];
    }
  }
  return 0;
}

int orc_nbins(const orc_params* p) { return (int)ceil(p->Lz / p->bin_width); }

int orc_observables(const orc_params* p, const orc_pore* pores, int npores, int64_t n,
                    const double* x, const double* d2wall, int64_t* occupancy, int64_t* adsorbed,
                    int64_t* profile, int nbins) {
  const int ngroups = npores > 0 ? npores : 1;
  if (nbins < orc_nbins(p)) return -1;
  for (int g = 0; g < npores; ++g) occupancy[g] = 0;
  for (int g = 0; g < ngroups; ++g) adsorbed[g] = 0;
  for (int64_t b = 0; b < (int64_t)ngroups * nbins; ++b) profile[b] = 0;
  const int nb = orc_nbins(p);
  for (int64_t i = 0; i < n; ++i) {
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    int g = 0;
    double best = INFINITY;
    for (int q = 0; q < npores; ++q) {
      double dx = min_image(xi - pores[q].cx, p->Lx), dy = min_image(yi - pores[q].cy, p->Ly);
      double d2 = pores[q].kind == 3 ? dy * dy : dx * dx + dy * dy;
      if (d2 < best) {
        best = d2;
        g = q;
      }
      if (fabs(zi) < p->slab_half && in_pore(&pores[q], dx, dy, zi, p->slab_half)) occupancy[q] += 1;
    }
    if (d2wall && d2wall[i] < p->r_ads * p->r_ads) adsorbed[g] += 1;
    int b = (int)floor((zi + 0.5 * p->Lz) / p->bin_width);
    if (b < 0) b = 0;
    if (b >= nb) b = nb - 1;
    profile[(int64_t)g * nbins + b] += 1;
  }
  return 0;
}

/* cross-section of a pore's carved region at height z: an area, or for dims == 2 a length in x */
static double pore_area(const orc_params* p, const orc_pore* q, double z) {
  const double h = p->slab_half;
  if (q->kind == 5) {
    if (z < prism_floor(q, h)) return 0.0; /* (the floor itself has measure zero) */
    return p->dims == 2 ? 2.0 * q->r0 : 4.0 * q->r0 * q->r1;
  }
  switch (q->kind) {
    case 1: return M_PI * q->r0 * q->r0;
    case 2: {
      double R = q->r0 + (q->r1 - q->r0) * (z + h) / (2.0 * h);
      return M_PI * R * R;
    }
    case 3: return q->width * p->Lx;
    case 4: {
      double c = q->r_cavity * q->r_cavity - z * z;
      double n2 = q->r0 * q->r0;
      return M_PI * (c > n2 ? c : n2);
    }
    default: return 0.0;
  }
}

double orc_pore_volume(const orc_params* p, const orc_pore* q) {
  const int m = 20000; /* even */
  double a = -p->slab_half;
  const double b = p->slab_half;
  if (q->kind == 5 && prism_floor(q, b) > a) a = prism_floor(q, b); /* where the pore is */
  const double step = (b - a) / m;
  double s = pore_area(p, q, a) + pore_area(p, q, b);
  for (int k = 1; k < m; ++k) s += (k % 2 ? 4.0 : 2.0) * pore_area(p, q, a + k * step);
  return s * step / 3.0;
}

int orc_pore_pressure(const orc_params* p, const orc_pore* pores, int npores, int64_t n,
                      const double* x, const double* v, const double* wvir, double* pressure) {
  for (int q = 0; q < npores; ++q) {
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double zi = x[3 * i + 2];
      if (!(fabs(zi) < p->slab_half)) continue;
      double dx = min_image(x[3 * i] - pores[q].cx, p->Lx);
      double dy = min_image(x[3 * i + 1] - pores[q].cy, p->Ly);
      if (!in_pore(&pores[q], dx, dy, zi, p->slab_half)) continue;
      sum += p->mass * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
      sum += wvir[i];
    }
    const double vol = orc_pore_volume(p, &pores[q]);
    pressure[q] = vol > 0.0 ? sum / ((p->dims == 2 ? 2.0 : 3.0) * vol) : 0.0;
  }
  return 0;
}
