/*
 * Plain FP64 CPU oracle of the UGKS step on a global adaptive velocity space
 * (arXiv 2212.05645).  TEST INFRASTRUCTURE ONLY: it is called by the tests,
 * by the smoke check and by the benchmark's CPU-baseline leg, never by the
 * product path.  It shares no code with the CUDA library.
 *
 * Layouts
 *   f      : [cell][array][node], array 0 = G, array 1 = H (2D only); with the
 *            Rykov model a last array R (rotational energy)
 *   Wc     : conserved variables per cell: rho, rho*U (D), rho*E; with the
 *            Rykov model also rho*E_rot
 *   Wp     : primitive variables per cell: rho, U (D), T
 *   xi     : [node][D] velocity-mesh node (element centre), w : [node] weight
 *   mesh   : face list, see om_mesh
 */
#ifndef AVS_ORACLE_H
#define AVS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int D, Nc, Nf, nbc;
    const int *faceL, *faceR;     /* faceR < 0: boundary condition -1-faceR */
    const double *An;             /* [Nf][D] area * unit normal, L -> R      */
    const double *rL, *rR;        /* [Nf][D] face centre - cell centre       */
    const double *vol;            /* [Nc]                                    */
    const double *bc;             /* [nbc][6] type, rho, U0, U1, U2, T       */
} om_mesh;

typedef struct {
    double R, Pr, omega, mu_ref, T_ref;
    double lim_K;                 /* Venkatakrishnan constant K              */
    int limiter;                  /* 0 first order, 1 Venkatakrishnan, 2 unlimited */
    int model;                    /* 0 Shakhov (monatomic), 1 Rykov (diatomic) */
    double Zrot, omega0, omega1, delta;   /* Rykov coefficients (Eqs. 11-13)  */
} om_gas;

enum { OM_COPY = 0, OM_MERGE = 1 };

double om_mu_ref_from_Kn(double Kn, double omega, double R);
void om_shakhov_field(int D, int Nv, const double *xi, double Pr, double rho, const double *U,
                      double RT, const double *q, double *gG, double *gH);

int  om_forest_base(int D, const int *nb, int *level, int *base, unsigned *key);
void om_forest_geom(int D, const int *nb, const double *vlo, const double *vhi, int Nv,
                    const int *level, const int *base, const unsigned *key,
                    double *xi, double *w);

void om_maxwell_init(int D, int Nc, int Nv, const double *xi, const double *Wp, double R,
                     double amp, unsigned long long seed, double *f);
void om_normal_field(unsigned long long seed, int Nc, int Nv, double *z);

void om_moments(int D, int Nc, int Nv, const double *xi, const double *w, const double *f,
                double *Wc, double *q);
double om_dt_unit(const om_mesh *m, int Nv, const double *xi);
/* step 1 of om_step alone: unlimited LSQ gradient grad [Nc][nA][Nv][D] and
 * Venkatakrishnan factor lim [Nc][nA][Nv] (Sec. 2.3.3) */
void om_limited_gradients(const om_mesh *m, const om_gas *g, int Nv, const double *f_in, double *grad, double *lim);
/* Venkatakrishnan's function of (largest neighbour difference, unlimited
 * change, epsilon^2), capped at 1 */
double om_venkat(double d1, double d2, double eps2);
int  om_step(const om_mesh *m, const om_gas *g, int Nv, const double *xi, const double *w,
             double dt, const double *f_in, double *f_out, double *Wc);

int  om_colors(const om_mesh *m, int *color);
int  om_step_implicit(const om_mesh *m, const om_gas *g, int Nv, const double *xi, const double *w,
                      double dt, const double *f_in, double *f_out, double *Wc,
                      const int *color, int ncolor, int k_macro, int k_micro);

void om_criterion(int D, int Nc, int Nv, const double *xi, const double *w, const double *f,
                  const double *Wc, double *M);
int  om_adapt_tree(int D, int Nv, const int *level, const int *base, const unsigned *key,
                   const double *M, double s, double C1, double C2, int max_refine, const int *lcap, int cap,
                   int *nlevel, int *nbase, unsigned *nkey, int *src, int *kind);
void om_remap(int D, int Nc, int Nv_old, const double *f_old, int Nv_new,
              const int *src, const int *kind, double *f_new);
double om_correct(int D, int Nc, int Nv, const double *xi, const double *w, double R,
                  int iters, const double *Wc_target, double *f);

/* Rykov model (diatomic gas, K = 2 rotational degrees of freedom) */
void om_rykov_field(int D, int Nv, const double *xi, const om_gas *g, double rho, const double *U,
                    double RTt, double RTr, const double *qt, const double *qr, double *out);
void om_maxwell_init_rykov(int D, int Nc, int Nv, const double *xi, const double *Wp, double R,
                           double amp, unsigned long long seed, double *f);
void om_moments_rykov(int D, int Nc, int Nv, const double *xi, const double *w, const double *f,
                      double *Wc, double *qt, double *qr);
void om_criterion_nw(int D, int nA, int nw, int Nc, int Nv, const double *xi, const double *w,
                     const double *f, const double *Wc, double *M);
void om_remap_n(int D, int nA, int Nc, int Nv_old, const double *f_old, int Nv_new,
                const int *src, const int *kind, double *f_new);
double om_correct_rykov(int D, int Nc, int Nv, const double *xi, const double *w, double R,
                        int iters, const double *Wc_target, double *f);

#ifdef __cplusplus
}
#endif
#endif
