/*
 * cg_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).  See cg_oracle.h.
 *
 * Plain FP64, one cell at a time, written from the paper's Sec. II:
 *   Sec. II.A  moments, harmonic relaxation time, Eq. (feq), Eq. (collision), Eq. (perturb),
 *              Eq. (cg) with its isotropic stencil, Eq. (recolor), Eq. (Stream);
 *   Sec. II.B  Eq. (relation) phi = S-bar varphi dx, Eq. (exchange), the site criterion
 *              |F| > Gamma using |F| of the previous step, and the six-step method summary.
 * Results III (first paragraph): halfway bounce-back walls, neutrally wetting.
 *
 * The lattice weights A_i, B_i, C_i, W_i and zeta are not printed in the paper (it defers them
 * to Leclaire et al. 2017); the values below are the standard ones of that model and are checked
 * by brute-force identities in tests/test_oracle_lattice.py.  Points the paper leaves open are
 * read as follows here:
 *   - a neighbour that is solid contributes rho^N of the evaluating cell to the gradient
 *     (neutral wetting);
 *   - cos(theta_i) of the recoloring term is 0 for the rest direction and where |F| = 0;
 *   - the perturbation vanishes where |F| = 0;
 *   - f^{b*} = f - f^{r*};
 *   - site rule "band" (|rho^N| < theta on the post-streaming, pre-exchange phase field) is
 *     offered besides the paper's gradient rule; ties are not sites (strict inequalities);
 *   - site rule "given" replays a recorded site set x_I (one mask per step), so that a
 *     derivative with respect to phi can be taken with x_I held fixed.
 */
#include "cg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19

typedef struct {
  int Q;
  int c[QMAX][3];
  double w[QMAX], a[QMAX], b[QMAX], cw[QMAX];
  double zeta;
  int opp[QMAX];
} lattice;

/* D2Q9: rest, 4 axis, 4 diagonal; opposite directions are adjacent (1<->2, 3<->4, ...). */
static const int C9[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
/* D3Q19: rest, 6 axis, 12 face diagonals. */
static const int C19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                               {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                               {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
                               {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};

static int make_lattice(int q, lattice *L) {
  const int(*c)[3];
  double w[3], a[3], b[3], cw[3];
  if (q == 9) {
    c = C9;
    /* |c|^2 = 0, 1, 2 */
    w[0] = 4.0 / 9.0;   w[1] = 1.0 / 9.0;   w[2] = 1.0 / 36.0;
    a[0] = 0.0;         a[1] = 1.0 / 5.0;   a[2] = 1.0 / 20.0;
    b[0] = 1.0;         b[1] = -1.0 / 5.0;  b[2] = -1.0 / 20.0;
    cw[0] = -4.0 / 27.0; cw[1] = 2.0 / 27.0; cw[2] = 5.0 / 108.0;
    L->zeta = 3.0 / 5.0;
  } else if (q == 19) {
    c = C19;
    w[0] = 1.0 / 3.0;   w[1] = 1.0 / 18.0;  w[2] = 1.0 / 36.0;
    a[0] = 0.0;         a[1] = 1.0 / 12.0;  a[2] = 1.0 / 24.0;
    b[0] = 1.0;         b[1] = -1.0 / 12.0; b[2] = -1.0 / 24.0;
    cw[0] = -1.0 / 3.0; cw[1] = 1.0 / 18.0; cw[2] = 1.0 / 36.0;
    L->zeta = 1.0 / 2.0;
  } else {
    return 0;
  }
  L->Q = q;
  for (int i = 0; i < q; i++) {
    int s = 0;
    for (int d = 0; d < 3; d++) {
      L->c[i][d] = c[i][d];
      s += c[i][d] * c[i][d];
    }
    L->w[i] = w[s];
    L->a[i] = a[s];
    L->b[i] = b[s];
    L->cw[i] = cw[s];
  }
  for (int i = 0; i < q; i++) {
    L->opp[i] = -1;
    for (int j = 0; j < q; j++)
      if (c[j][0] == -c[i][0] && c[j][1] == -c[i][1] && c[j][2] == -c[i][2]) L->opp[i] = j;
  }
  return q;
}

int orc_lattice(int q, int *c, double *w, double *a, double *b, double *cw, double *zeta,
                int *opp) {
  lattice L;
  if (!make_lattice(q, &L)) return 0;
  for (int i = 0; i < q; i++) {
    for (int d = 0; d < 3; d++) c[3 * i + d] = L.c[i][d];
    w[i] = L.w[i];
    a[i] = L.a[i];
    b[i] = L.b[i];
    cw[i] = L.cw[i];
    opp[i] = L.opp[i];
  }
  *zeta = L.zeta;
  return q;
}

/* Sec. II.A: the least dense component gets alpha = W_0; any other one gets
 * 1 - (1 - W_0) / gamma_k with gamma_k = rho_k_in / rho_min_in. */
void orc_alphas(const orc_params *p, double *alpha_r, double *alpha_b) {
  lattice L;
  make_lattice(p->q, &L);
  double w0 = L.w[0];
  double rmin = p->rho_r_in < p->rho_b_in ? p->rho_r_in : p->rho_b_in;
  *alpha_r = (p->rho_r_in <= rmin) ? w0 : 1.0 - (1.0 - w0) / (p->rho_r_in / rmin);
  *alpha_b = (p->rho_b_in <= rmin) ? w0 : 1.0 - (1.0 - w0) / (p->rho_b_in / rmin);
}

static void feq_on(const lattice *L, double rho, const double *u, double abar, double *feq) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < L->Q; i++) {
    double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    feq[i] = rho * (L->a[i] + L->b[i] * abar + L->w[i] * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
  }
}

static void perturbation_on(const lattice *L, const double *F, double *out) {
  double Fn = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  for (int i = 0; i < L->Q; i++) {
    if (Fn == 0.0) {
      out[i] = 0.0;
      continue;
    }
    double Fc = F[0] * L->c[i][0] + F[1] * L->c[i][1] + F[2] * L->c[i][2];
    out[i] = Fn * (L->w[i] * Fc * Fc / (Fn * Fn) - L->cw[i]);
  }
}

void orc_feq(int q, double rho, const double *u, double abar, double *feq) {
  lattice L;
  if (make_lattice(q, &L)) feq_on(&L, rho, u, abar, feq);
}

void orc_perturbation_shape(int q, const double *F, double *out) {
  lattice L;
  if (make_lattice(q, &L)) perturbation_on(&L, F, out);
}

/* ---------------------------------------------------------------- geometry -------------- */

/* The wall-normal axis of the outlets: z in 3D, y in 2D. */
static int normal_axis(const orc_params *p) { return p->q == 19 ? 2 : 1; }

static int valid_params(const orc_params *p) {
  if (!p) return 0;
  if ((p->outlet_rho_lo > 0.0 || p->outlet_rho_hi > 0.0) && p->periodic[normal_axis(p)]) return 0;
  if (p->q != 9 && p->q != 19) return 0;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return 0;
  if (p->q == 9 && p->nz != 1) return 0;
  if (p->tau_r <= 0.5 || p->tau_b <= 0.5) return 0;
  if (p->rho_r_in <= 0.0 || p->rho_b_in <= 0.0) return 0;
  if (p->beta < 0.0 || p->beta > 1.0) return 0;
  if (p->sbar <= 0.0) return 0;
  if (p->site_rule == ORC_RULE_GIVEN && !p->mask_given) return 0;
  return 1;
}

static long long ncells(const orc_params *p) { return (long long)p->nx * p->ny * p->nz; }

static long long idx(const orc_params *p, int x, int y, int z) {
  return ((long long)z * p->ny + y) * p->nx + x;
}

static int is_solid(const orc_params *p, long long X) { return p->solid && p->solid[X]; }

/* Index of the cell at (x,y,z)+d, or -1 where that cell is solid or lies beyond a wall. */
static long long neighbour(const orc_params *p, int x, int y, int z, int dx, int dy, int dz) {
  int n[3] = {p->nx, p->ny, p->nz};
  int r[3] = {x + dx, y + dy, z + dz};
  for (int d = 0; d < 3; d++) {
    if (r[d] < 0 || r[d] >= n[d]) {
      if (!p->periodic[d]) return -1;
      r[d] = (r[d] % n[d] + n[d]) % n[d];
    }
  }
  long long Y = idx(p, r[0], r[1], r[2]);
  return is_solid(p, Y) ? -1 : Y;
}

/* -------------------------------------------------------------- per-cell pieces ----------- */

/* Eq. (Stream) in pull form: f_i^k(x) = f_i^{k*}(x - c_i); where x - c_i is solid the
 * population leaving x towards it comes back reversed (halfway bounce-back). */
/* Pressure outlet for the blue component (Sec. III.B.2; the boundary condition of Zou and He).
 * gb holds the blue populations of a cell on an outlet plane after the pull, n the inward
 * normal along `axis`.  The populations with c.n = +1 come from outside and are unknown; with
 * the blue density fixed at rho0 and no blue velocity along the plane:
 *   mass + normal momentum:  rho0 u_n = rho0 - (S_0 + 2 S_out),
 *       S_0 = sum over c.n = 0, S_out = sum over c.n = -1 (known populations);
 *   non-equilibrium bounce-back: g_i = g_opp(i) + (f_i^eq - f_opp(i)^eq) = g_opp(i) + 6 W_i rho0 u_n
 *       (only the odd part of Eq. feq differs between i and opp(i));
 *   tangential momentum zero: each tangential axis t gets -c_it N_t,
 *       N_t = (1/2) sum over c.n = 0 of g_j c_jt.
 * Red populations keep their bounce-back values: the outlet lets no red through. */
static void outlet_blue(const lattice *L, int axis, int inward, double rho0, double gb[QMAX]) {
  double s0 = 0.0, sout = 0.0, t[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < L->Q; i++) {
    int cn = L->c[i][axis] * inward;
    if (cn == 0) {
      s0 += gb[i];
      for (int d = 0; d < 3; d++)
        if (d != axis) t[d] += L->c[i][d] * gb[i];
    } else if (cn < 0) {
      sout += gb[i];
    }
  }
  double un = 1.0 - (s0 + 2.0 * sout) / rho0;
  for (int i = 0; i < L->Q; i++) {
    if (L->c[i][axis] * inward <= 0) continue;
    double corr = 0.0;
    for (int d = 0; d < 3; d++)
      if (d != axis) corr += L->c[i][d] * 0.5 * t[d];
    gb[i] = gb[L->opp[i]] + 6.0 * L->w[i] * rho0 * un - corr;
  }
}

static void pull_cell(const orc_params *p, const lattice *L, const double *f_in, int x, int y,
                      int z, double g[2][QMAX]) {
  long long N = ncells(p), X = idx(p, x, y, z);
  for (int i = 0; i < L->Q; i++) {
    long long S = neighbour(p, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
    for (int k = 0; k < 2; k++) {
      if (S < 0)
        g[k][i] = f_in[((long long)k * L->Q + L->opp[i]) * N + X];
      else
        g[k][i] = f_in[((long long)k * L->Q + i) * N + S];
    }
  }
  int ax = normal_axis(p);
  int r[3] = {x, y, z}, n[3] = {p->nx, p->ny, p->nz};
  if (p->outlet_rho_lo > 0.0 && r[ax] == 0) outlet_blue(L, ax, +1, p->outlet_rho_lo, g[1]);
  if (p->outlet_rho_hi > 0.0 && r[ax] == n[ax] - 1) outlet_blue(L, ax, -1, p->outlet_rho_hi, g[1]);
}

static void densities(const lattice *L, double g[2][QMAX], double *rr, double *rb) {
  double a = 0.0, b = 0.0;
  for (int i = 0; i < L->Q; i++) {
    a += g[0][i];
    b += g[1][i];
  }
  *rr = a;
  *rb = b;
}

/* Steps 2 and 3 of the method summary for one cell: decide whether it is an evaporation site
 * and, if so, move varphi = phi/S-bar from the red to the blue rest population (Eq. exchange).
 * Returns the site flag; *margin is the distance of the decision value from the threshold. */
static int select_and_exchange(const orc_params *p, const lattice *L, double g[2][QMAX],
                               const double *G_prev, long long X, double *margin,
                               double *moved) {
  int site;
  if (p->site_rule == ORC_RULE_GIVEN) {
    /* the site set of an earlier run, replayed: Eq. (exchange) with x_I held fixed */
    site = p->mask_given[X] & 1;
    *margin = INFINITY;
  } else if (p->site_rule == ORC_RULE_GRADIENT) {
    double G = G_prev ? G_prev[X] : 0.0;
    site = G > p->threshold;
    *margin = fabs(G - p->threshold);
  } else {
    double rr, rb;
    densities(L, g, &rr, &rb);
    double rn = (rr - rb) / (rr + rb);
    site = fabs(rn) < p->threshold;
    *margin = fabs(fabs(rn) - p->threshold);
  }
  *moved = 0.0;
  if (site) {
    double phi = p->phi_field ? p->phi_field[X] : p->phi;
    double varphi = phi / p->sbar; /* Eq. (relation) */
    g[0][0] -= varphi;
    g[1][0] += varphi;
    *moved = varphi;
  }
  return site;
}

/* Eq. (cg) with the isotropic stencil: F = (1/cs^2) sum_i W_i rho^N(x + c_i) c_i. */
static void color_gradient(const lattice *L, const double rn_nb[QMAX], double F[3]) {
  F[0] = F[1] = F[2] = 0.0;
  for (int i = 0; i < L->Q; i++)
    for (int d = 0; d < 3; d++) F[d] += 3.0 * L->w[i] * rn_nb[i] * L->c[i][d];
}

/* Step 4 (moments) and step 5 (collision, perturbation, recoloring) for one cell. */
static void collide_cell(const orc_params *p, const lattice *L, double alpha_r, double alpha_b,
                         double g[2][QMAX], const double F[3], double out[2][QMAX]) {
  int Q = L->Q;
  double rr, rb;
  densities(L, g, &rr, &rb);
  double rho = rr + rb;
  double f[QMAX], u[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; i++) {
    f[i] = g[0][i] + g[1][i]; /* colour-blind population */
    for (int d = 0; d < 3; d++) u[d] += f[i] * L->c[i][d];
  }
  for (int d = 0; d < 3; d++) u[d] /= rho;
  double wr = rr / rho, wb = rb / rho;
  double inv_tau = wr / p->tau_r + wb / p->tau_b; /* harmonic average of tau_k */
  double abar = wr * alpha_r + wb * alpha_b;

  double feq[QMAX];
  feq_on(L, rho, u, abar, feq);
  for (int i = 0; i < Q; i++) f[i] = f[i] - inv_tau * (f[i] - feq[i]); /* Eq. (collision) */

  double shape[QMAX];
  perturbation_on(L, F, shape);
  for (int i = 0; i < Q; i++) f[i] += 2.25 * p->sigma * inv_tau * shape[i]; /* Eq. (perturb) */

  double Fn = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  for (int i = 0; i < Q; i++) { /* Eq. (recolor) */
    double cosv = 0.0;
    if (i != 0 && Fn > 0.0) {
      double Fc = F[0] * L->c[i][0] + F[1] * L->c[i][1] + F[2] * L->c[i][2];
      double cn = sqrt((double)(L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] +
                                L->c[i][2] * L->c[i][2]));
      cosv = Fc / (Fn * cn);
    }
    double feq_rest = rho * (L->a[i] + L->b[i] * abar); /* f_i^eq(rho, 0) */
    out[0][i] = wr * f[i] + p->beta * wr * wb * cosv * feq_rest;
    out[1][i] = f[i] - out[0][i];
  }
}

/* ------------------------------------------------------------------ public -------------- */

int orc_init(const orc_params *p, const double *rhoN0, const double *noise, double *f) {
  if (!valid_params(p)) return -1;
  lattice L;
  make_lattice(p->q, &L);
  double ar, ab;
  orc_alphas(p, &ar, &ab);
  long long N = ncells(p);
  for (long long X = 0; X < N; X++) {
    double rk[2] = {p->rho_r_in * (1.0 + rhoN0[X]) / 2.0, p->rho_b_in * (1.0 - rhoN0[X]) / 2.0};
    double al[2] = {ar, ab};
    for (int k = 0; k < 2; k++)
      for (int i = 0; i < L.Q; i++) {
        long long o = ((long long)k * L.Q + i) * N + X;
        if (is_solid(p, X)) {
          f[o] = 0.0;
          continue;
        }
        f[o] = rk[k] * (L.a[i] + L.b[i] * al[k]) + (noise ? noise[o] : 0.0);
      }
  }
  return 0;
}

/* rho^N from the local sums of a state (Sec. II.A). */
static void local_rhoN(const orc_params *p, const lattice *L, const double *f, double *rn) {
  long long N = ncells(p);
  for (long long X = 0; X < N; X++) {
    if (is_solid(p, X)) {
      rn[X] = 0.0;
      continue;
    }
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < L->Q; i++) {
      rr += f[(long long)i * N + X];
      rb += f[((long long)L->Q + i) * N + X];
    }
    rn[X] = (rr - rb) / (rr + rb);
  }
}

static void gather_rn(const orc_params *p, const lattice *L, const double *rn, int x, int y,
                      int z, double rn_nb[QMAX]) {
  long long X = idx(p, x, y, z);
  for (int i = 0; i < L->Q; i++) {
    long long Y = neighbour(p, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
    rn_nb[i] = (Y < 0) ? rn[X] : rn[Y];
  }
}

int orc_gradient_norm(const orc_params *p, const double *f, double *G) {
  if (!valid_params(p)) return -1;
  lattice L;
  make_lattice(p->q, &L);
  long long N = ncells(p);
  double *rn = (double *)malloc(sizeof(double) * N);
  if (!rn) return -2;
  local_rhoN(p, &L, f, rn);
  for (int z = 0; z < p->nz; z++)
    for (int y = 0; y < p->ny; y++)
      for (int x = 0; x < p->nx; x++) {
        long long X = idx(p, x, y, z);
        if (is_solid(p, X)) {
          G[X] = 0.0;
          continue;
        }
        double nb[QMAX], F[3];
        gather_rn(p, &L, rn, x, y, z, nb);
        color_gradient(&L, nb, F);
        G[X] = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
      }
  free(rn);
  return 0;
}

int orc_step(const orc_params *p, const double *f_in, double *f_out, const double *G_prev,
             double *G_out, unsigned char *mask_out, double *margin_out, orc_ledger *led) {
  if (!valid_params(p)) return -1;
  if (p->site_rule == ORC_RULE_GRADIENT && !G_prev) return -1;
  lattice L;
  make_lattice(p->q, &L);
  double ar, ab;
  orc_alphas(p, &ar, &ab);
  int Q = L.Q;
  long long N = ncells(p);
  double *g = (double *)malloc(sizeof(double) * 2 * Q * N);
  double *rn = (double *)malloc(sizeof(double) * N);
  if (!g || !rn) {
    free(g);
    free(rn);
    return -2;
  }

  /* Streaming, Eq. (Stream), pull form.  (The omp pragmas only matter in the separately built
     timing library of the CPU baseline; the pinned oracle is compiled without OpenMP.) */
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < p->nz; z++)
    for (int y = 0; y < p->ny; y++)
      for (int x = 0; x < p->nx; x++) {
        long long X = idx(p, x, y, z);
        if (is_solid(p, X)) continue;
        double gc[2][QMAX];
        pull_cell(p, &L, f_in, x, y, z, gc);
        for (int k = 0; k < 2; k++)
          for (int i = 0; i < Q; i++) g[((long long)k * Q + i) * N + X] = gc[k][i];
      }

  /* Steps 1-3: sink rate, site selection, exchange of rest populations. */
  long long sites = 0;
  double removed = 0.0, min_margin = INFINITY;
#pragma omp parallel for schedule(static) reduction(+ : sites, removed) reduction(min : min_margin)
  for (long long X = 0; X < N; X++) {
    if (is_solid(p, X)) {
      mask_out[X] = 0;
      if (margin_out) margin_out[X] = INFINITY;
      continue;
    }
    double gc[2][QMAX];
    for (int k = 0; k < 2; k++)
      for (int i = 0; i < Q; i++) gc[k][i] = g[((long long)k * Q + i) * N + X];
    double margin, moved;
    int site = select_and_exchange(p, &L, gc, G_prev, X, &margin, &moved);
    g[0 * N + X] = gc[0][0];
    g[(long long)Q * N + X] = gc[1][0];
    mask_out[X] = (unsigned char)site;
    if (margin_out) margin_out[X] = margin;
    if (margin < min_margin) min_margin = margin;
    if (site) {
      sites++;
      removed += moved;
    }
  }

  /* Step 4: moments of every cell, needed by the gradient stencil. */
#pragma omp parallel for schedule(static)
  for (long long X = 0; X < N; X++) {
    if (is_solid(p, X)) {
      rn[X] = 0.0;
      continue;
    }
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < Q; i++) {
      rr += g[(long long)i * N + X];
      rb += g[((long long)Q + i) * N + X];
    }
    rn[X] = (rr - rb) / (rr + rb);
  }

  /* Step 5: colour gradient, collision, perturbation, recoloring. */
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < p->nz; z++)
    for (int y = 0; y < p->ny; y++)
      for (int x = 0; x < p->nx; x++) {
        long long X = idx(p, x, y, z);
        if (is_solid(p, X)) {
          for (int k = 0; k < 2; k++)
            for (int i = 0; i < Q; i++) f_out[((long long)k * Q + i) * N + X] = 0.0;
          if (G_out) G_out[X] = 0.0;
          continue;
        }
        double nb[QMAX], F[3], gc[2][QMAX], out[2][QMAX];
        gather_rn(p, &L, rn, x, y, z, nb);
        color_gradient(&L, nb, F);
        for (int k = 0; k < 2; k++)
          for (int i = 0; i < Q; i++) gc[k][i] = g[((long long)k * Q + i) * N + X];
        collide_cell(p, &L, ar, ab, gc, F, out);
        for (int k = 0; k < 2; k++)
          for (int i = 0; i < Q; i++) f_out[((long long)k * Q + i) * N + X] = out[k][i];
        if (G_out) G_out[X] = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
      }

  if (led) {
    led->evaporated += removed;
    led->site_steps += sites;
    led->last_sites = sites;
    led->last_removed = removed;
    led->min_margin = min_margin;
  }
  free(g);
  free(rn);
  return 0;
}

/* rho^N of cell (x,y,z) after streaming and exchange, computed on its own. */
static double rn_after_exchange(const orc_params *p, const lattice *L, const double *f_in,
                                const double *G_prev, int x, int y, int z) {
  double g[2][QMAX], margin, moved, rr, rb;
  pull_cell(p, L, f_in, x, y, z, g);
  select_and_exchange(p, L, g, G_prev, idx(p, x, y, z), &margin, &moved);
  densities(L, g, &rr, &rb);
  return (rr - rb) / (rr + rb);
}

int orc_step_cells(const orc_params *p, const double *f_in, const double *G_prev,
                   const long long *cells, long long ncells_, double *out_f, double *out_G,
                   unsigned char *out_mask) {
  if (!valid_params(p)) return -1;
  if (p->site_rule == ORC_RULE_GRADIENT && !G_prev) return -1;
  lattice L;
  make_lattice(p->q, &L);
  double ar, ab;
  orc_alphas(p, &ar, &ab);
  int Q = L.Q;
  long long N = ncells(p);
  for (long long s = 0; s < ncells_; s++) {
    long long X = cells[s];
    if (X < 0 || X >= N) return -1;
    int x = (int)(X % p->nx), y = (int)((X / p->nx) % p->ny), z = (int)(X / ((long long)p->nx * p->ny));
    double *o = out_f + s * 2 * Q;
    if (is_solid(p, X)) {
      for (int j = 0; j < 2 * Q; j++) o[j] = 0.0;
      out_G[s] = 0.0;
      out_mask[s] = 0;
      continue;
    }
    double g[2][QMAX], margin, moved;
    pull_cell(p, &L, f_in, x, y, z, g);
    out_mask[s] = (unsigned char)select_and_exchange(p, &L, g, G_prev, X, &margin, &moved);
    double rr, rb;
    densities(&L, g, &rr, &rb);
    double own = (rr - rb) / (rr + rb);
    double nb[QMAX], F[3], out[2][QMAX];
    for (int i = 0; i < Q; i++) {
      long long Y = neighbour(p, x, y, z, L.c[i][0], L.c[i][1], L.c[i][2]);
      if (Y < 0) {
        nb[i] = own;
      } else {
        int yx = (int)(Y % p->nx), yy = (int)((Y / p->nx) % p->ny),
            yz = (int)(Y / ((long long)p->nx * p->ny));
        nb[i] = rn_after_exchange(p, &L, f_in, G_prev, yx, yy, yz);
      }
    }
    color_gradient(&L, nb, F);
    collide_cell(p, &L, ar, ab, g, F, out);
    for (int k = 0; k < 2; k++)
      for (int i = 0; i < Q; i++) o[k * Q + i] = out[k][i];
    out_G[s] = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
  }
  return 0;
}

int orc_outlet_blue(int q, int inward, double rho0, double *gb) {
  lattice L;
  if (!make_lattice(q, &L) || (inward != 1 && inward != -1) || !(rho0 > 0.0)) return -1;
  double g[QMAX];
  for (int i = 0; i < L.Q; i++) g[i] = gb[i];
  outlet_blue(&L, q == 19 ? 2 : 1, inward, rho0, g);
  for (int i = 0; i < L.Q; i++) gb[i] = g[i];
  return 0;
}

int orc_macros(const orc_params *p, const double *f, double *rho_r, double *rho_b, double *u,
               double *rhoN) {
  if (!valid_params(p)) return -1;
  lattice L;
  make_lattice(p->q, &L);
  long long N = ncells(p);
  for (long long X = 0; X < N; X++) {
    double rr = 0.0, rb = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L.Q; i++) {
      double fr = f[(long long)i * N + X], fb = f[((long long)L.Q + i) * N + X];
      rr += fr;
      rb += fb;
      for (int d = 0; d < 3; d++) j[d] += (fr + fb) * L.c[i][d];
    }
    double rho = rr + rb;
    if (rho_r) rho_r[X] = rr;
    if (rho_b) rho_b[X] = rb;
    for (int d = 0; d < 3; d++)
      if (u) u[(long long)d * N + X] = (rho > 0.0) ? j[d] / rho : 0.0;
    if (rhoN) rhoN[X] = (rho > 0.0) ? (rr - rb) / rho : 0.0;
  }
  return 0;
}
