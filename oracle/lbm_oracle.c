/*
 * FP64 CPU oracle for the elastic-wall D3Q19 lattice Boltzmann step of
 * McCullough & Coveney, "An efficient, localised approach for the simulation
 * of elastic blood vessels using the lattice Boltzmann method" (2021).
 *
 * TEST INFRASTRUCTURE ONLY.  The product library never links, imports or
 * calls anything in this directory; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * It is deliberately plain:
 *   - its own lattice builder from the voxel labels (integer, canonical order),
 *   - populations f[site][19] in array-of-structures order, two buffers (A-B),
 *   - one pass per step: moments -> equilibrium -> BGK collision -> push along
 *     each of the 18 links, with the boundary rule applied where the link
 *     leaves the fluid,
 *   - all arithmetic in double, compiled with -ffp-contract=off so the rounding
 *     follows the order written here.
 *
 * Passages followed (section / equation of the paper):
 *   Sec. 2.1: D3Q19 velocity set and weights; Eq. (LBE_SRT) single-relaxation
 *     update; Eq. (feq) equilibrium (read with the factors 1/2 of the standard
 *     second-order expansion, see equilibrium() below); Eqs. (Density),
 *     (Momentum) moments; Eq. (Pressure) p = c_s^2 rho.
 *   Sec. 2.3: Guo-Zheng-Shi extrapolation wall with Delta = 1 and the elastic
 *     wall velocity U_w = (F + dr - dx)/dr * U_f.
 *   Sec. 2.4: tube law dE = (1 - sigma^2) R^2/(Y h) (p - P0), folded into one
 *     per-wall-site stiffness kappa (lattice units), and the rigid bounce-back
 *     comparison.
 *   Sec. 3: velocity-profile inlet and fixed-pressure outlets.
 *
 * Readings taken where the paper is silent or garbled (each one is listed with
 * its reason in the design notes of the repository):
 *   R1 equilibrium carries the 1/2 factors;
 *   R2 dr = dx + dE (distance from the fluid node to the displaced wall);
 *   R3 dE is clamped at zero for p < P0 (fluid nodes are the minimum volume);
 *   R4 p - P0 = c_s^2 (rho_f - rho0);
 *   R5 link length dx = 1 for all 18 links;
 *   R6 U_w scales the full velocity vector u_f;
 *   R7 the wall uses the pre-collision moments of the fluid site at step n;
 *   R8 inlets: GZS form with (rho_f, u_in(x, n)); outlets: GZS form with
 *      (rho_out, u_f).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* Sec. 2.1: the rest vector, the 6 axis vectors and the 12 face diagonals, in
 * the order 0 rest; 1/2 +-x; 3/4 +-y; 5/6 +-z; 7/8 (+1,+1,0)/(-1,-1,0);
 * 9/10 (+1,-1,0)/(-1,+1,0); 11/12 (+1,0,+1)/(-1,0,-1); 13/14 (+1,0,-1)/(-1,0,+1);
 * 15/16 (0,+1,+1)/(0,-1,-1); 17/18 (0,+1,-1)/(0,-1,+1). */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

/* Sec. 2.1: weights 1/3 (rest), 1/18 (axes), 1/36 (diagonals); c_s^2 = 1/3. */
static double weight(int i) {
  if (i == 0) return 1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* The direction whose velocity is -c_i, found by search. */
static int opposite(int i) {
  for (int j = 0; j < Q; ++j)
    if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) return j;
  return -1;
}

typedef struct orc_iolet {
  int32_t kind;    /* 0 velocity inlet, 1 fixed-density outlet */
  int32_t profile; /* inlet shape: 0 parabolic, 1 rigid Womersley, 2 plug */
  double rho;      /* outlet density */
  double u_mean, u_amp, period, phase;
  double centre[3], axis[3], radius;
} orc_iolet;

typedef struct orc_lattice {
  int32_t nx, ny, nz, n_iolets;
  int64_t n;             /* fluid sites */
  int32_t *xyz;          /* [n][3] */
  int64_t *nbr;          /* [n][Q]: >= 0 fluid site, -1 wall, -2-k iolet k */
  int64_t n_wall;        /* sites with at least one wall link */
  int64_t *wall_site;    /* [n_wall] ascending */
  int64_t *wall_of_site; /* [n] wall index or -1 */
  int64_t n_wall_links;
  /* configuration */
  double tau, rho0;
  int32_t wall_model; /* 0 bounce-back, 1 elastic GZS */
  double *F, *kappa;  /* [n_wall] */
  orc_iolet *iolets;  /* [n_iolets] */
  double *alpha;      /* [n_iolets] Womersley number of each inlet */
  /* state */
  double *f, *fn; /* [n][Q] */
  int64_t step;
  double *dE, *Uw; /* [n_wall], [n_wall][3] from the most recent step */
} orc_lattice;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

void orc_free(orc_lattice *L) {
  if (!L) return;
  free(L->xyz); free(L->nbr); free(L->wall_site); free(L->wall_of_site);
  free(L->F); free(L->kappa); free(L->iolets); free(L->alpha);
  free(L->f); free(L->fn); free(L->dE); free(L->Uw);
  free(L);
}

/* Site order: ascending (x*ny + y)*nz + z, i.e. z fastest.  Link class: a
 * neighbour outside the box or labelled 0 is a wall; label 1 is fluid; label
 * 2+k is the ghost node of iolet k. */
int orc_build(const uint8_t *labels, int32_t nx, int32_t ny, int32_t nz, int32_t n_iolets,
              orc_lattice **out) {
  *out = NULL;
  if (nx <= 0 || ny <= 0 || nz <= 0 || n_iolets < 0 || n_iolets > 253) return ORC_EINVAL;
  int64_t nvox = (int64_t)nx * ny * nz;
  for (int64_t v = 0; v < nvox; ++v)
    if (labels[v] > 1 + n_iolets) return ORC_EINVAL;
  orc_lattice *L = (orc_lattice *)calloc(1, sizeof(orc_lattice));
  if (!L) return ORC_ENOMEM;
  L->nx = nx; L->ny = ny; L->nz = nz; L->n_iolets = n_iolets;
  int64_t *site_of_voxel = (int64_t *)malloc(sizeof(int64_t) * nvox);
  if (!site_of_voxel) { orc_free(L); return ORC_ENOMEM; }
  int64_t n = 0;
  for (int64_t v = 0; v < nvox; ++v) site_of_voxel[v] = labels[v] == 1 ? n++ : -1;
  L->n = n;
  L->xyz = (int32_t *)malloc(sizeof(int32_t) * 3 * (n ? n : 1));
  L->nbr = (int64_t *)malloc(sizeof(int64_t) * Q * (n ? n : 1));
  L->wall_of_site = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  if (!L->xyz || !L->nbr || !L->wall_of_site) { free(site_of_voxel); orc_free(L); return ORC_ENOMEM; }
  for (int32_t x = 0; x < nx; ++x)
    for (int32_t y = 0; y < ny; ++y)
      for (int32_t z = 0; z < nz; ++z) {
        int64_t s = site_of_voxel[((int64_t)x * ny + y) * nz + z];
        if (s < 0) continue;
        L->xyz[3 * s] = x; L->xyz[3 * s + 1] = y; L->xyz[3 * s + 2] = z;
        for (int i = 0; i < Q; ++i) {
          int32_t X = x + CX[i], Y = y + CY[i], Z = z + CZ[i];
          int64_t code;
          if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) {
            code = -1;
          } else {
            int64_t v = ((int64_t)X * ny + Y) * nz + Z;
            uint8_t lab = labels[v];
            if (lab == 0) code = -1;
            else if (lab == 1) code = site_of_voxel[v];
            else code = -2 - (int64_t)(lab - 2);
          }
          L->nbr[Q * s + i] = code;
        }
      }
  free(site_of_voxel);
  int64_t nw = 0, nl = 0;
  for (int64_t s = 0; s < n; ++s) {
    int walls = 0;
    for (int i = 1; i < Q; ++i) walls += L->nbr[Q * s + i] == -1;
    L->wall_of_site[s] = walls ? nw++ : -1;
    nl += walls;
  }
  L->n_wall = nw;
  L->n_wall_links = nl;
  L->wall_site = (int64_t *)malloc(sizeof(int64_t) * (nw ? nw : 1));
  L->F = (double *)calloc(nw ? nw : 1, sizeof(double));
  L->kappa = (double *)calloc(nw ? nw : 1, sizeof(double));
  L->dE = (double *)calloc(nw ? nw : 1, sizeof(double));
  L->Uw = (double *)calloc(3 * (nw ? nw : 1), sizeof(double));
  L->f = (double *)calloc((size_t)Q * (n ? n : 1), sizeof(double));
  L->fn = (double *)calloc((size_t)Q * (n ? n : 1), sizeof(double));
  L->iolets = (orc_iolet *)calloc(n_iolets ? n_iolets : 1, sizeof(orc_iolet));
  L->alpha = (double *)calloc(n_iolets ? n_iolets : 1, sizeof(double));
  if (!L->wall_site || !L->F || !L->kappa || !L->dE || !L->Uw || !L->f || !L->fn || !L->iolets ||
      !L->alpha) {
    orc_free(L);
    return ORC_ENOMEM;
  }
  for (int64_t s = 0; s < n; ++s)
    if (L->wall_of_site[s] >= 0) L->wall_site[L->wall_of_site[s]] = s;
  L->tau = 1.0; L->rho0 = 1.0; L->wall_model = 0;
  *out = L;
  return ORC_OK;
}

int64_t orc_n_sites(const orc_lattice *L) { return L->n; }
int64_t orc_n_wall_sites(const orc_lattice *L) { return L->n_wall; }
int64_t orc_n_wall_links(const orc_lattice *L) { return L->n_wall_links; }
int64_t orc_step_count(const orc_lattice *L) { return L->step; }

/* coords [n][3]; nbr [n][18] for directions 1..18; wall_sites [n_wall];
 * wall_links [n_wall_links][2] = (site, direction), sorted by (site, dir). */
void orc_export(const orc_lattice *L, int32_t *coords, int64_t *nbr, int64_t *wall_sites,
                int64_t *wall_links) {
  int64_t k = 0;
  for (int64_t s = 0; s < L->n; ++s) {
    if (coords) for (int d = 0; d < 3; ++d) coords[3 * s + d] = L->xyz[3 * s + d];
    for (int i = 1; i < Q; ++i) {
      int64_t c = L->nbr[Q * s + i];
      if (nbr) nbr[18 * s + (i - 1)] = c;
      if (c == -1 && wall_links) { wall_links[2 * k] = s; wall_links[2 * k + 1] = i; ++k; }
    }
  }
  if (wall_sites) for (int64_t w = 0; w < L->n_wall; ++w) wall_sites[w] = L->wall_site[w];
}

/* Complex Bessel functions J0, J1 by their power series
 *   J_n(z) = sum_k (-1)^k (z/2)^(2k+n) / (k! (k+n)!),
 * summed until the term falls below 1e-17 of the running sum.  Good to about
 * 1e-12 relative for |z| <= 12 and 1e-9 for |z| <= 20 (cancellation). */
static void bessel_j01(double complex z, double complex *j0, double complex *j1) {
  double complex h = z / 2.0, h2 = h * h;
  double complex t0 = 1.0, t1 = h, s0 = 0.0, s1 = 0.0;
  for (int k = 0; k < 200; ++k) {
    s0 += t0; s1 += t1;
    t0 *= -h2 / ((double)(k + 1) * (double)(k + 1));
    t1 *= -h2 / ((double)(k + 1) * (double)(k + 2));
    if (cabs(t0) < 1e-17 * cabs(s0) && cabs(t1) < 1e-17 * cabs(s1) && k > 2) break;
  }
  *j0 = s0; *j1 = s1;
}

void orc_bessel_j01(double re, double im, double *j0, double *j1) {
  double complex a, b;
  bessel_j01(re + im * I, &a, &b);
  j0[0] = creal(a); j0[1] = cimag(a);
  j1[0] = creal(b); j1[1] = cimag(b);
}

/* Rigid-tube Womersley profile of the oscillatory part (Sec. 2.2, the axial
 * velocity with M = 1 and c -> infinity), normalised to a unit mean over the
 * disc:  s(xi) = (1 - J0(L xi)/J0(L)) / (1 - 2 J1(L)/(L J0(L))),
 * L = i^(3/2) alpha, xi = r/R.  As alpha -> 0 it tends to 2 (1 - xi^2). */
static double complex womersley_shape(double alpha, double xi) {
  if (alpha < 1e-6) return 2.0 * (1.0 - xi * xi);
  double complex lam = alpha * cexp(I * 3.0 * M_PI / 4.0);
  double complex j0L, j1L, j0r, j1r;
  bessel_j01(lam, &j0L, &j1L);
  bessel_j01(lam * xi, &j0r, &j1r);
  double complex num = 1.0 - j0r / j0L;
  double complex den = 1.0 - 2.0 * j1L / (lam * j0L);
  return num / den;
}

void orc_womersley_shape(double alpha, double xi, double *s) {
  double complex v = womersley_shape(alpha, xi);
  s[0] = creal(v); s[1] = cimag(v);
}

/* Eq. (Viscosity): nu = c_s^2 (tau - 1/2); Womersley number alpha = R sqrt(omega/nu). */
int orc_configure(orc_lattice *L, double tau, int32_t wall_model, double rho0, const double *F,
                  const double *kappa, int64_t n_params, const orc_iolet *iolets,
                  int32_t n_iolets) {
  if (!(tau > 0.5) || (wall_model != 0 && wall_model != 1) || n_iolets != L->n_iolets)
    return ORC_EINVAL;
  if (n_params != 1 && n_params != L->n_wall && L->n_wall > 0) return ORC_EINVAL;
  L->tau = tau; L->wall_model = wall_model; L->rho0 = rho0;
  for (int64_t w = 0; w < L->n_wall; ++w) {
    double Fw = F ? F[n_params == 1 ? 0 : w] : 0.0;
    double kw = kappa ? kappa[n_params == 1 ? 0 : w] : 0.0;
    if (!(Fw >= 0.0) || !(kw >= 0.0) || !isfinite(Fw) || !isfinite(kw)) return ORC_EINVAL;
    L->F[w] = Fw; L->kappa[w] = kw;
  }
  double nu = (tau - 0.5) / 3.0;
  for (int k = 0; k < n_iolets; ++k) {
    orc_iolet io = iolets[k];
    if (io.kind != 0 && io.kind != 1) return ORC_EINVAL;
    double an = sqrt(io.axis[0] * io.axis[0] + io.axis[1] * io.axis[1] + io.axis[2] * io.axis[2]);
    if (!(an > 0.0)) return ORC_EINVAL;
    for (int d = 0; d < 3; ++d) io.axis[d] /= an;
    L->iolets[k] = io;
    L->alpha[k] = io.period > 0.0 ? io.radius * sqrt(2.0 * M_PI / io.period / nu) : 0.0;
  }
  return ORC_OK;
}

/* Eq. (feq) with c_s^2 = 1/3 and the standard factors 1/2:
 *   f_i^eq = w_i rho (1 + c.u/c_s^2 + (c.u)^2/(2 c_s^4) - u.u/(2 c_s^2)). */
static double equilibrium(int i, double rho, const double u[3]) {
  double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Eqs. (Density), (Momentum). */
static void moments(const double *f, double *rho, double u[3]) {
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < Q; ++i) {
    r += f[i];
    jx += f[i] * CX[i]; jy += f[i] * CY[i]; jz += f[i] * CZ[i];
  }
  *rho = r;
  u[0] = jx / r; u[1] = jy / r; u[2] = jz / r;
}

void orc_velocity_set(int32_t *c, double *w, int32_t *opp) {
  for (int i = 0; i < Q; ++i) {
    if (c) { c[3 * i] = CX[i]; c[3 * i + 1] = CY[i]; c[3 * i + 2] = CZ[i]; }
    if (w) w[i] = weight(i);
    if (opp) opp[i] = opposite(i);
  }
}

void orc_equilibrium(double rho, const double *u, double *feq) {
  for (int i = 0; i < Q; ++i) feq[i] = equilibrium(i, rho, u);
}

/* Eq. (LBE_SRT) without the streaming: f* = f - (f - f^eq)/tau. */
void orc_collide(const double *f, double tau, double *out) {
  double rho, u[3];
  moments(f, &rho, u);
  for (int i = 0; i < Q; ++i) out[i] = f[i] - (f[i] - equilibrium(i, rho, u)) / tau;
}

/* Inlet velocity at fluid site s and step n: u_in = a (u_mean p0(r) +
 * u_amp (ps(r) sin(theta) + pc(r) cos(theta))), theta = 2 pi n / T + phase,
 * with (p0, ps, pc) the shape of the chosen profile and r the distance from the
 * inlet axis (the profile is evaluated at the fluid site). */
static void inlet_velocity(const orc_lattice *L, int k, int64_t s, int64_t n, double ub[3]) {
  const orc_iolet *io = &L->iolets[k];
  double d[3], along = 0.0, dd = 0.0;
  for (int c = 0; c < 3; ++c) {
    d[c] = (double)L->xyz[3 * s + c] - io->centre[c];
    along += d[c] * io->axis[c];
    dd += d[c] * d[c];
  }
  double r2 = dd - along * along;
  double q = r2 / (io->radius * io->radius);
  double p0, ps, pc;
  if (io->profile == 2) {
    p0 = 1.0; ps = 1.0; pc = 0.0;
  } else {
    p0 = q < 1.0 ? 2.0 * (1.0 - q) : 0.0;
    ps = p0; pc = 0.0;
    if (io->profile == 1) {
      if (q < 1.0) {
        double complex sh = womersley_shape(L->alpha[k], sqrt(q > 0.0 ? q : 0.0));
        ps = creal(sh); pc = cimag(sh);
      } else {
        ps = 0.0; pc = 0.0;
      }
    }
  }
  double g = io->u_mean * p0;
  if (io->period > 0.0) {
    double theta = 2.0 * M_PI * (double)n / io->period + io->phase;
    g += io->u_amp * (ps * sin(theta) + pc * cos(theta));
  }
  for (int c = 0; c < 3; ++c) ub[c] = g * io->axis[c];
}

/* One step of Eq. (LBE_SRT) over all sites, with the boundary rules. */
static void step_once(orc_lattice *L, int nthreads) {
  const double tau = L->tau;
  const double dx = 1.0; /* R5: link length dx for every link */
  const int64_t n = L->n, nstep = L->step;
  double *f = L->f, *fn = L->fn;
  int opp[Q];
  for (int i = 0; i < Q; ++i) opp[i] = opposite(i);
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t x = 0; x < n; ++x) {
    const double *fx = f + (size_t)Q * x;
    const int64_t *nb = L->nbr + (size_t)Q * x;
    double rho, u[3], feq[Q], fneq[Q], fstar[Q];
    moments(fx, &rho, u);
    for (int i = 0; i < Q; ++i) {
      feq[i] = equilibrium(i, rho, u);
      fneq[i] = fx[i] - feq[i];
      fstar[i] = fx[i] - fneq[i] / tau;
    }
    /* Sec. 2.3/2.4: wall velocity from the local pressure (R2-R4, R6, R7). */
    double Uw[3] = {0.0, 0.0, 0.0};
    int64_t w = L->wall_of_site[x];
    if (w >= 0) {
      double p = (rho - L->rho0) / 3.0;        /* c_s^2 (rho - rho0) */
      double dE = L->kappa[w] * (p > 0.0 ? p : 0.0);
      double dr = dx + dE;
      double scale = (L->F[w] + dr - dx) / dr; /* U_w = (F + dr - dx)/dr U_f */
      for (int c = 0; c < 3; ++c) Uw[c] = scale * u[c];
      L->dE[w] = dE;
      for (int c = 0; c < 3; ++c) L->Uw[3 * w + c] = Uw[c];
    }
    for (int i = 0; i < Q; ++i) {
      int64_t y = i == 0 ? x : nb[i];
      if (y >= 0) {
        fn[(size_t)Q * y + i] = fstar[i];
        continue;
      }
      int j = opp[i];
      double val;
      if (y == -1) {
        if (L->wall_model == 0) {
          val = fstar[i]; /* half-way bounce-back */
        } else {
          val = equilibrium(j, rho, Uw) + (1.0 - 1.0 / tau) * fneq[j];
        }
      } else {
        int k = (int)(-2 - y);
        const orc_iolet *io = &L->iolets[k];
        if (io->kind == 0) {
          double ub[3];
          inlet_velocity(L, k, x, nstep, ub);
          val = equilibrium(j, rho, ub) + (1.0 - 1.0 / tau) * fneq[j];
        } else {
          val = equilibrium(j, io->rho, u) + (1.0 - 1.0 / tau) * fneq[j];
        }
      }
      fn[(size_t)Q * x + j] = val;
    }
  }
  L->f = fn;
  L->fn = f;
  L->step = nstep + 1;
}

int orc_run(orc_lattice *L, int64_t n_steps, int32_t nthreads) {
  if (n_steps < 0) return ORC_EINVAL;
  for (int64_t s = 0; s < n_steps; ++s) step_once(L, nthreads);
  return ORC_OK;
}

/* f = f^eq(rho, u) per site; NULL rho means 1, NULL u means 0. Resets the step counter. */
void orc_init_equilibrium(orc_lattice *L, const double *rho, const double *u) {
  for (int64_t s = 0; s < L->n; ++s) {
    double r = rho ? rho[s] : 1.0;
    double v[3] = {0.0, 0.0, 0.0};
    if (u) { v[0] = u[3 * s]; v[1] = u[3 * s + 1]; v[2] = u[3 * s + 2]; }
    for (int i = 0; i < Q; ++i) L->f[(size_t)Q * s + i] = equilibrium(i, r, v);
  }
  L->step = 0;
}

void orc_set_populations(orc_lattice *L, const double *f, int64_t step) {
  memcpy(L->f, f, sizeof(double) * Q * (size_t)L->n);
  L->step = step;
}

void orc_get_populations(const orc_lattice *L, double *f) {
  memcpy(f, L->f, sizeof(double) * Q * (size_t)L->n);
}

void orc_moments(const orc_lattice *L, double *rho, double *u) {
  for (int64_t s = 0; s < L->n; ++s) {
    double r, v[3];
    moments(L->f + (size_t)Q * s, &r, v);
    if (rho) rho[s] = r;
    if (u) { u[3 * s] = v[0]; u[3 * s + 1] = v[1]; u[3 * s + 2] = v[2]; }
  }
}

void orc_wall_state(const orc_lattice *L, double *dE, double *Uw) {
  for (int64_t w = 0; w < L->n_wall; ++w) {
    if (dE) dE[w] = L->dE[w];
    if (Uw) for (int c = 0; c < 3; ++c) Uw[3 * w + c] = L->Uw[3 * w + c];
  }
}

/* out[0] = total mass sum_x rho_x; out[1 + k] = sum over sites with a link into
 * iolet k of (rho u) . axis_k, the mass flux through the first fluid layer. */
void orc_reduce(const orc_lattice *L, double *out) {
  double mass = 0.0;
  for (int k = 0; k < L->n_iolets; ++k) out[1 + k] = 0.0;
  for (int64_t s = 0; s < L->n; ++s) {
    const double *fx = L->f + (size_t)Q * s;
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
      r += fx[i];
      j[0] += fx[i] * CX[i]; j[1] += fx[i] * CY[i]; j[2] += fx[i] * CZ[i];
    }
    mass += r;
    for (int k = 0; k < L->n_iolets; ++k) {
      int touches = 0;
      for (int i = 1; i < Q; ++i) touches |= L->nbr[(size_t)Q * s + i] == -2 - k;
      if (touches) {
        const double *a = L->iolets[k].axis;
        out[1 + k] += j[0] * a[0] + j[1] * a[1] + j[2] * a[2];
      }
    }
  }
  out[0] = mass;
}

/* Wall shear stress at the given sites (reading of the paper's WSS fields,
 * which it does not define): deviatoric stress
 *   sigma = -(1 - 1/(2 tau)) sum_i f_i^neq c_i c_i,
 * traction t = sigma n with the given outward unit normal n, and
 * WSS = |t - (t.n) n|.  Uses the current (pre-collision) populations. */
void orc_wss(const orc_lattice *L, const int64_t *sites, const double *normals, int64_t m,
             double *out) {
  for (int64_t q = 0; q < m; ++q) {
    const double *fx = L->f + (size_t)Q * sites[q];
    double rho, u[3], P[3][3] = {{0}};
    moments(fx, &rho, u);
    for (int i = 0; i < Q; ++i) {
      double fneq = fx[i] - equilibrium(i, rho, u);
      int c[3] = {CX[i], CY[i], CZ[i]};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) P[a][b] += fneq * c[a] * c[b];
    }
    const double *nv = normals + 3 * q;
    double t[3], tn = 0.0;
    for (int a = 0; a < 3; ++a) {
      t[a] = 0.0;
      for (int b = 0; b < 3; ++b) t[a] += -(1.0 - 1.0 / (2.0 * L->tau)) * P[a][b] * nv[b];
    }
    for (int a = 0; a < 3; ++a) tn += t[a] * nv[a];
    double s2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double ta = t[a] - tn * nv[a];
      s2 += ta * ta;
    }
    out[q] = sqrt(s2);
  }
}
