/*
 * cg_oracle.h -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * Plain, slow, FP64 CPU statement of one timestep of the two-component color-gradient (CG)
 * lattice Boltzmann model with the reaction-limited (RL) evaporation step of Nath, Aouane and
 * Harting, "Reaction-limited evaporation for the color-gradient lattice Boltzmann model"
 * (arXiv:2412.14859).  Only tests/, __graft_entry__.smoke() and the CPU-baseline legs of
 * bench.py may load it.  It shares no source, header, table or helper with the CUDA library.
 *
 * State convention.  The stored state is the post-recoloring population f_i^{k*}(x) of the last
 * completed step, laid out as double f[k][i][z][y][x] (k = 0 red, 1 blue; x fastest).  One call
 * of orc_step performs the streaming of Eq. (Stream) (pull form) followed by steps 1-5 of the
 * method summary at the end of Sec. II.B.  Solid cells hold zeros and are never updated.
 */
#ifndef CG_ORACLE_H
#define CG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_RULE_GRADIENT 0  /* site if |F| of the previous step > threshold (Sec. II.B)        */
#define ORC_RULE_BAND     1  /* site if |rho^N| of the current step < threshold (phase band)    */
#define ORC_RULE_GIVEN    2  /* site where bit 0 of mask_given is set (a replayed site set)     */

typedef struct {
  int q;                 /* 9 (D2Q9, nz must be 1) or 19 (D3Q19)                                */
  int nx, ny, nz;
  int periodic[3];       /* 1 periodic, 0 = halfway bounce-back walls just outside both ends    */
  double rho_r_in, rho_b_in;  /* initial bulk densities; alpha_k follow Sec. II.A               */
  double tau_r, tau_b;   /* component relaxation times                                          */
  double sigma;          /* surface tension in Eq. (perturb)                                    */
  double beta;           /* recoloring parameter of Eq. (recolor)                               */
  int site_rule;         /* ORC_RULE_GRADIENT, ORC_RULE_BAND or ORC_RULE_GIVEN                  */
  double threshold;      /* Gamma (gradient rule) or theta (band rule)                          */
  double sbar;           /* S-bar of Eq. (relation)                                             */
  double phi;            /* flux, used when phi_field is NULL                                   */
  const double *phi_field;        /* per-cell flux [z][y][x] or NULL                            */
  const unsigned char *solid;     /* per-cell solid flag [z][y][x] or NULL                      */
  const unsigned char *mask_given; /* ORC_RULE_GIVEN: sites are the cells whose bit 0 is set     */
  /* Blue pressure outlets (Sec. III.B.2) on the first / last plane of the wall-normal axis (z in
   * 3D, y in 2D, which must have walls): the prescribed blue density there, or <= 0 for a wall. */
  double outlet_rho_lo, outlet_rho_hi;
} orc_params;

typedef struct {
  double evaporated;     /* cumulative sum over steps and sites of varphi = phi / S-bar         */
  long long site_steps;  /* cumulative number of (site, step) pairs                             */
  long long last_sites;  /* number of sites at the last step                                    */
  double last_removed;   /* mass moved red -> blue at the last step                             */
  double min_margin;     /* smallest |decision value - threshold| over fluid cells, last step   */
} orc_ledger;

/* Lattice tables; returns Q or 0 for an unsupported q. */
int orc_lattice(int q, int *c /* [Q][3] */, double *w, double *a, double *b, double *cw,
                double *zeta, int *opp);

/* alpha_r, alpha_b from the initial densities (Sec. II.A). */
void orc_alphas(const orc_params *p, double *alpha_r, double *alpha_b);

/* Equilibrium of Eq. (feq) for one cell: feq[i] = rho [A_i + B_i abar + W_i (...)]. */
void orc_feq(int q, double rho, const double *u, double abar, double *feq);

/* Perturbation term of Eq. (perturb) for unit amplitude: out[i] = |F|[W_i (F.c_i)^2/|F|^2 - C_i]. */
void orc_perturbation_shape(int q, const double *F, double *out);

/* f_i^k = rho_k phi_i(alpha_k) + noise, rho_r = rho_r_in (1+rhoN0)/2, rho_b = rho_b_in (1-rhoN0)/2. */
int orc_init(const orc_params *p, const double *rhoN0, const double *noise, double *f);

/* |F| of the state f (local densities), used as the "previous step" |F| before step 0. */
int orc_gradient_norm(const orc_params *p, const double *f, double *G);

/* One timestep.  G_prev: |F| of the previous step (gradient rule; may be NULL for the band rule).
 * Writes f_out, G_out (|F| of this step), mask_out (1 where a site), margin_out (per-cell
 * |decision value - threshold|, may be NULL) and updates the ledger.  Returns 0 on success. */
int orc_step(const orc_params *p, const double *f_in, double *f_out, const double *G_prev,
             double *G_out, unsigned char *mask_out, double *margin_out, orc_ledger *led);

/* The same step evaluated only at the listed cells (linear indices); out_f is [ncells][2][Q],
 * out_G [ncells], out_mask [ncells].  Used to check single outputs of very large lattices. */
int orc_step_cells(const orc_params *p, const double *f_in, const double *G_prev,
                   const long long *cells, long long ncells, double *out_f, double *out_G,
                   unsigned char *out_mask);

/* The blue outlet of one cell on its own: gb [Q] are the pulled blue populations of a cell on
 * the first (inward = +1) or last (inward = -1) plane of the wall-normal axis; the populations
 * entering from outside are replaced as the step does for an outlet of blue density rho0. */
int orc_outlet_blue(int q, int inward, double rho0, double *gb);

/* Local macroscopic fields of the state: rho_r, rho_b, u (3 x N) and rho^N. */
int orc_macros(const orc_params *p, const double *f, double *rho_r, double *rho_b, double *u,
               double *rhoN);

#ifdef __cplusplus
}
#endif
#endif
