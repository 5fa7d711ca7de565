/*
 * Plain FP64 CPU oracle of the explicit UGKS step on a global adaptive
 * velocity space (arXiv 2212.05645).  TEST INFRASTRUCTURE: only the tests,
 * the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Every routine follows the paper's definitions in the paper's order, with
 * plain loops (cells, then arrays, then nodes; faces in list order) and no
 * blocking or fusion.  Where the paper is silent, the comment beside the code
 * states the reading taken (tagged R1..R32 so that the tests can name it).
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include "avs_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXS 8            /* face slots per cell */
#define PI 3.14159265358979323846

static int nArr(int D) { return D == 2 ? 2 : 1; }

/* ---- gas model ----------------------------------------------------------- */

/* Eq. (4)-(5) with rho = T = L_ref = 1:  Kn = 2 mu (5-2w)(7-2w) / (15 sqrt(2 pi R)) */
double om_mu_ref_from_Kn(double Kn, double omega, double R)
{
    return 15.0 * sqrt(2.0 * PI * R) * Kn / (2.0 * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega));
}

/* Eq. (3): tau = mu / (rho R T), VHS mu = mu_ref (T / T_ref)^omega */
static double tau_of(const om_gas *g, double rho, double RT)
{
    double T = RT / g->R;
    double mu = g->mu_ref * pow(T / g->T_ref, g->omega);
    return mu / (rho * RT);
}

/* conserved -> rho, U, RT.  Monatomic gas: rho E = rho U^2 / 2 + (3/2) rho R T
 * (three translational degrees of freedom, K = 0; Eq. 7). */
static void prim_of(int D, const double *Wc, double *rho, double *U, double *RT)
{
    double r = Wc[0];
    double m2 = 0.0;
    for (int d = 0; d < D; ++d) {
        U[d] = Wc[1 + d] / r;
        m2 += Wc[1 + d] * Wc[1 + d];
    }
    *rho = r;
    *RT = (Wc[D + 1] - 0.5 * m2 / r) / (1.5 * r);
}

/* Eq. (Maxwell_df): g = rho / (2 pi R T)^(D/2) exp(-|xi-U|^2 / (2 R T)) */
static double maxwell(int D, double rho, const double *U, double RT, const double *xi)
{
    double c2 = 0.0;
    for (int d = 0; d < D; ++d) c2 += (xi[d] - U[d]) * (xi[d] - U[d]);
    return rho / pow(2.0 * PI * RT, 0.5 * D) * exp(-c2 / (2.0 * RT));
}

/* Eqs. (14)-(17), monatomic (K = 0): Shakhov equilibrium of the reduced
 * distributions.  The second line of Eq. (14) is read as g^H. */
static void shakhov(int D, double Pr, double rho, const double *U, double RT, const double *q,
                    const double *xi, double *gG, double *gH)
{
    double c[3], c2 = 0.0, cq = 0.0;
    for (int d = 0; d < D; ++d) {
        c[d] = xi[d] - U[d];
        c2 += c[d] * c[d];
        cq += c[d] * q[d];
    }
    double geq = rho / pow(2.0 * PI * RT, 0.5 * D) * exp(-c2 / (2.0 * RT));
    double p = rho * RT;
    double a = (1.0 - Pr) * cq / (5.0 * p * RT);
    *gG = geq + a * (c2 / RT - D - 2.0) * geq;                       /* g^eq + G_Pr */
    double Heq = (3.0 - D) * RT * geq;                               /* Eq. 16      */
    *gH = Heq + a * ((c2 / RT - D) * (3.0 - D)) * RT * geq;          /* + H_Pr      */
}

/* ---- Rykov model (diatomic gas; Sec. 2.1, Eqs. updat_W, 8, GHR_equ, 11-13) ----
 * Reduced distributions: G, H, R in 2D and G, R in 3D (H carries the
 * 3 - D dummy translational components and vanishes for D = 3; reading R23).
 * W = (rho, rho U, rho E, rho E_rot) with rho E = int (xi^2 G + H)/2 + R and
 * rho E_rot = int R.  With K = 2 rotational degrees of freedom (R24):
 * rho E_rot = rho R T_r, (3/2) rho R T_t = rho E - rho U^2/2 - rho E_rot and
 * the equilibrium temperature T = (3 T_t + 2 T_r) / 5. */
static int nArrG(const om_gas *g, int D) { return g->model ? (D == 2 ? 3 : 2) : nArr(D); }
static int nWG(const om_gas *g, int D) { return g->model ? D + 3 : D + 2; }

static void prim_rykov(int D, const double *Wc, double *rho, double *U, double *RTt, double *RTr, double *RT)
{
    double r = Wc[0];
    double m2 = 0.0;
    for (int d = 0; d < D; ++d) {
        U[d] = Wc[1 + d] / r;
        m2 += Wc[1 + d] * Wc[1 + d];
    }
    *rho = r;
    *RTr = Wc[D + 2] / r;
    *RTt = (Wc[D + 1] - 0.5 * m2 / r - Wc[D + 2]) / (1.5 * r);
    *RT = (Wc[D + 1] - 0.5 * m2 / r) / (2.5 * r);
}

/* Rykov equilibrium at one node (Eqs. GHR_equ, 11-13): out[0] = g^G,
 * out[1] = g^H (2D), out[nA - 1] = g^R. */
static void rykov(int D, const om_gas *g, double rho, const double *U, double RTt, double RTr,
                  const double *qt, const double *qr, const double *xi, double *out)
{
    double c[3], c2 = 0.0, cqt = 0.0, cqr = 0.0;
    for (int d = 0; d < D; ++d) {
        c[d] = xi[d] - U[d];
        c2 += c[d] * c[d];
        cqt += c[d] * qt[d];
        cqr += c[d] * qr[d];
    }
    double RT = (3.0 * RTt + 2.0 * RTr) / 5.0;
    double gt = maxwell(D, rho, U, RTt, xi);
    double gr = maxwell(D, rho, U, RT, xi);
    double pt = rho * RTt, p = rho * RT;
    double at = cqt / (15.0 * pt * RTt);
    double ar = g->omega0 * cqt / (15.0 * p * RT);
    double Gt = gt * (1.0 + at * (c2 / RTt - D - 2.0));
    double Gr = gr * (1.0 + ar * (c2 / RT - D - 2.0));
    double Ht = RTt * gt * (3.0 - D) * (1.0 + at * (c2 / RTt - D));
    double Hr = RT * gr * (3.0 - D) * (1.0 + ar * (c2 / RT - D));
    double Rt = RTr * (Gt + (1.0 - g->delta) * cqr / (pt * RTt) * gt);
    double Rr = RT * (Gr + g->omega1 * (1.0 - g->delta) * cqr / (p * RT) * gr);
    double iz = 1.0 / g->Zrot;
    out[0] = (1.0 - iz) * Gt + iz * Gr;
    if (D == 2) out[1] = (1.0 - iz) * Ht + iz * Hr;
    out[D == 2 ? 2 : 1] = (1.0 - iz) * Rt + iz * Rr;
}

void om_rykov_field(int D, int Nv, const double *xi, const om_gas *g, double rho, const double *U,
                    double RTt, double RTr, const double *qt, const double *qr, double *out)
{
    int nA = D == 2 ? 3 : 2;
    for (int k = 0; k < Nv; ++k) {
        double v[3];
        rykov(D, g, rho, U, RTt, RTr, qt, qr, xi + (size_t)k * D, v);
        for (int a = 0; a < nA; ++a) out[(size_t)a * Nv + k] = v[a];
    }
}

/* Moments (Eqs. updat_W, 8): W = (rho, rho U, rho E, rho E_rot); about U,
 * q_t = int c (c^2 G + H) / 2 and q_r = int c R. */
static void cell_moments_rykov(int D, int Nv, const double *xi, const double *w, const double *fi,
                               double *Wc, double *qt, double *qr)
{
    const double *G = fi, *H = D == 2 ? fi + Nv : NULL, *Rr = fi + (size_t)(D == 2 ? 2 : 1) * Nv;
    double rho = 0.0, m[3] = {0, 0, 0}, E = 0.0, Er = 0.0;
    for (int k = 0; k < Nv; ++k) {
        const double *x = xi + (size_t)k * D;
        double x2 = 0.0;
        for (int d = 0; d < D; ++d) x2 += x[d] * x[d];
        rho += w[k] * G[k];
        for (int d = 0; d < D; ++d) m[d] += w[k] * x[d] * G[k];
        E += w[k] * (0.5 * (x2 * G[k] + (H ? H[k] : 0.0)) + Rr[k]);
        Er += w[k] * Rr[k];
    }
    Wc[0] = rho;
    for (int d = 0; d < D; ++d) Wc[1 + d] = m[d];
    Wc[D + 1] = E;
    Wc[D + 2] = Er;
    if (qt || qr) {
        double U[3], a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) U[d] = m[d] / rho;
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double c[3], c2 = 0.0;
            for (int d = 0; d < D; ++d) {
                c[d] = x[d] - U[d];
                c2 += c[d] * c[d];
            }
            for (int d = 0; d < D; ++d) {
                a[d] += 0.5 * w[k] * c[d] * (c2 * G[k] + (H ? H[k] : 0.0));
                b[d] += w[k] * c[d] * Rr[k];
            }
        }
        for (int d = 0; d < D; ++d) {
            if (qt) qt[d] = a[d];
            if (qr) qr[d] = b[d];
        }
    }
}

void om_moments_rykov(int D, int Nc, int Nv, const double *xi, const double *w, const double *f,
                      double *Wc, double *qt, double *qr)
{
    int nA = D == 2 ? 3 : 2;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Nc; ++i)
        cell_moments_rykov(D, Nv, xi, w, f + (size_t)i * nA * Nv, Wc + (size_t)i * (D + 3),
                           qt ? qt + (size_t)i * D : NULL, qr ? qr + (size_t)i * D : NULL);
}

/* Shakhov equilibrium (G, H) of one state at every node; exported for tests. */
void om_shakhov_field(int D, int Nv, const double *xi, double Pr, double rho, const double *U,
                      double RT, const double *q, double *gG, double *gH)
{
    for (int k = 0; k < Nv; ++k) {
        double h;
        shakhov(D, Pr, rho, U, RT, q, xi + (size_t)k * D, gG + k, gH ? gH + k : &h);
    }
}

/* ---- velocity forest (Sec. 3.1) ---------------------------------------- */

/* Level-0 base forest, base cells in row-major order (axis 0 fastest). */
int om_forest_base(int D, const int *nb, int *level, int *base, unsigned *key)
{
    int n = 1;
    for (int d = 0; d < D; ++d) n *= nb[d];
    for (int b = 0; b < n; ++b) {
        level[b] = 0;
        base[b] = b;
        key[b] = 0u;
    }
    return n;
}

/* Mid-point quadrature (Sec. 3): node = element centre, weight = element
 * area/volume.  Path digits c = o0 | o1 << 1 | o2 << 2, most significant
 * digit = first refinement.  xi = vlo + hb * (b + (2 o + 1) / 2^(l+1)). */
void om_forest_geom(int D, const int *nb, const double *vlo, const double *vhi, int Nv,
                    const int *level, const int *base, const unsigned *key,
                    double *xi, double *w)
{
    double hb[3];
    for (int d = 0; d < D; ++d) hb[d] = (vhi[d] - vlo[d]) / (double)nb[d];
    for (int k = 0; k < Nv; ++k) {
        int l = level[k];
        int b = base[k];
        int bi[3];
        for (int d = 0; d < D; ++d) {
            bi[d] = b % nb[d];
            b /= nb[d];
        }
        double wk = 1.0;
        for (int d = 0; d < D; ++d) {
            unsigned o = 0;
            for (int m = 0; m < l; ++m) {
                unsigned digit = (key[k] >> (D * (l - 1 - m))) & ((1u << D) - 1u);
                o = 2u * o + ((digit >> d) & 1u);
            }
            double frac = (double)(2u * o + 1u) / (double)(1u << (l + 1));
            xi[k * D + d] = vlo[d] + hb[d] * ((double)bi[d] + frac);
            wk *= hb[d];
        }
        w[k] = ldexp(wk, -D * l);
    }
}

/* ---- synthetic initial field -------------------------------------------- */

static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double normal_ik(uint64_t seed, uint64_t i, uint64_t k)
{
    uint64_t key = (i << 32) | k;
    uint64_t u1 = splitmix64(seed ^ splitmix64(2u * key));
    uint64_t u2 = splitmix64(seed ^ splitmix64(2u * key + 1u));
    double U1 = ((double)(u1 >> 11) + 1.0) * 0x1p-53;
    double U2 = (double)(u2 >> 11) * 0x1p-53;
    return sqrt(-2.0 * log(U1)) * cos(2.0 * PI * U2);
}

void om_normal_field(unsigned long long seed, int Nc, int Nv, double *z)
{
    for (int i = 0; i < Nc; ++i)
        for (int k = 0; k < Nv; ++k) z[(size_t)i * Nv + k] = normal_ik(seed, (uint64_t)i, (uint64_t)k);
}

/* G = g^eq(W_i)(xi_k) (1 + amp z_ik), H = (3 - D) R T G  (Eq. 16, K = 0). */
void om_maxwell_init(int D, int Nc, int Nv, const double *xi, const double *Wp, double R,
                     double amp, unsigned long long seed, double *f)
{
    int nA = nArr(D);
    for (int i = 0; i < Nc; ++i) {
        const double *P = Wp + (size_t)i * (D + 2);
        double RT = R * P[D + 1];
        for (int k = 0; k < Nv; ++k) {
            double G = maxwell(D, P[0], P + 1, RT, xi + (size_t)k * D);
            if (amp != 0.0) G *= 1.0 + amp * normal_ik(seed, (uint64_t)i, (uint64_t)k);
            f[((size_t)i * nA + 0) * Nv + k] = G;
            if (nA == 2) f[((size_t)i * nA + 1) * Nv + k] = (3.0 - D) * RT * G;
        }
    }
}

/* Initial field: G = g^eq(rho, U, T_t)(1 + amp z_ik), H = (3 - D) R T_t G,
 * R = R T_r G.  Wp per cell: rho, U (D), T_t, T_r. */
void om_maxwell_init_rykov(int D, int Nc, int Nv, const double *xi, const double *Wp, double R,
                           double amp, unsigned long long seed, double *f)
{
    int nA = D == 2 ? 3 : 2;
    for (int i = 0; i < Nc; ++i) {
        const double *P = Wp + (size_t)i * (D + 3);
        double RTt = R * P[D + 1], RTr = R * P[D + 2];
        for (int k = 0; k < Nv; ++k) {
            double G = maxwell(D, P[0], P + 1, RTt, xi + (size_t)k * D);
            if (amp != 0.0) G *= 1.0 + amp * normal_ik(seed, (uint64_t)i, (uint64_t)k);
            f[((size_t)i * nA + 0) * Nv + k] = G;
            if (D == 2) f[((size_t)i * nA + 1) * Nv + k] = (3.0 - D) * RTt * G;
            f[((size_t)i * nA + nA - 1) * Nv + k] = RTr * G;
        }
    }
}

/* ---- moments (Eq. 7, Eq. 8) --------------------------------------------- */

static void cell_moments(int D, int Nv, const double *xi, const double *w, const double *fi,
                         double *Wc, double *q)
{
    int nA = nArr(D);
    const double *G = fi;
    const double *H = nA == 2 ? fi + Nv : NULL;
    double rho = 0.0, m[3] = {0, 0, 0}, E = 0.0;
    for (int k = 0; k < Nv; ++k) {
        const double *x = xi + (size_t)k * D;
        double x2 = 0.0;
        for (int d = 0; d < D; ++d) x2 += x[d] * x[d];
        rho += w[k] * G[k];
        for (int d = 0; d < D; ++d) m[d] += w[k] * x[d] * G[k];
        E += 0.5 * w[k] * (x2 * G[k] + (H ? H[k] : 0.0));
    }
    Wc[0] = rho;
    for (int d = 0; d < D; ++d) Wc[1 + d] = m[d];
    Wc[D + 1] = E;
    if (q) {
        double U[3];
        for (int d = 0; d < D; ++d) U[d] = m[d] / rho;
        double qq[3] = {0, 0, 0};
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double c[3], c2 = 0.0;
            for (int d = 0; d < D; ++d) {
                c[d] = x[d] - U[d];
                c2 += c[d] * c[d];
            }
            for (int d = 0; d < D; ++d) qq[d] += 0.5 * w[k] * c[d] * (c2 * G[k] + (H ? H[k] : 0.0));
        }
        for (int d = 0; d < D; ++d) q[d] = qq[d];
    }
}

void om_moments(int D, int Nc, int Nv, const double *xi, const double *w, const double *f,
                double *Wc, double *q)
{
    int nA = nArr(D);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < Nc; ++i)
        cell_moments(D, Nv, xi, w, f + (size_t)i * nA * Nv, Wc + (size_t)i * (D + 2),
                     q ? q + (size_t)i * D : NULL);
}

/* ---- cell -> face slots ------------------------------------------------- */

typedef struct {
    int n;
    int face[MAXS];
    int sgn[MAXS];   /* +1: cell is L (An points outward), -1: cell is R */
} slots_t;

static slots_t *build_slots(const om_mesh *m)
{
    slots_t *S = (slots_t *)calloc((size_t)m->Nc, sizeof(slots_t));
    for (int f = 0; f < m->Nf; ++f) {
        int L = m->faceL[f], R = m->faceR[f];
        slots_t *s = &S[L];
        s->face[s->n] = f;
        s->sgn[s->n] = +1;
        s->n++;
        if (R >= 0) {
            s = &S[R];
            s->face[s->n] = f;
            s->sgn[s->n] = -1;
            s->n++;
        }
    }
    return S;
}

/* offset from the centre of cell i to the centre of its face in slot s */
static const double *slot_r(const om_mesh *m, const slots_t *S, int i, int s)
{
    int f = S[i].face[s];
    return S[i].sgn[s] > 0 ? m->rL + (size_t)f * m->D : m->rR + (size_t)f * m->D;
}

static int slot_nb(const om_mesh *m, const slots_t *S, int i, int s)
{
    int f = S[i].face[s];
    return S[i].sgn[s] > 0 ? m->faceR[f] : m->faceL[f];
}

/* Δt from the CFL number (reading R5): min over cells and nodes of
 * |V_i| / sum_faces max(xi_k . An_out, 0).  Returns that minimum (Δt / CFL). */
double om_dt_unit(const om_mesh *m, int Nv, const double *xi)
{
    int D = m->D;
    slots_t *S = build_slots(m);
    double best = INFINITY;
    for (int i = 0; i < m->Nc; ++i) {
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double sum = 0.0;
            for (int s = 0; s < S[i].n; ++s) {
                const double *a = m->An + (size_t)S[i].face[s] * D;
                double sn = 0.0;
                for (int d = 0; d < D; ++d) sn += x[d] * a[d];
                sn *= S[i].sgn[s];
                if (sn > 0.0) sum += sn;
            }
            if (sum > 0.0) {
                double t = m->vol[i] / sum;
                if (t < best) best = t;
            }
        }
    }
    free(S);
    return best;
}

/* ---- least-squares gradient + Venkatakrishnan limiter (Sec. 2.3.3) ---- */

/* Inverse of the LSQ normal matrix sum w d d^T with weights 1/|d|^2 (R6).
 * Returns 0 when the matrix is singular (gradient taken as zero). */
static int lsq_inverse(const om_mesh *m, const slots_t *S, int i, double *Minv)
{
    int D = m->D;
    double M[9] = {0};
    for (int s = 0; s < S[i].n; ++s) {
        int nb = slot_nb(m, S, i, s);
        if (nb < 0) continue;
        int f = S[i].face[s];
        const double *rs = S[i].sgn[s] > 0 ? m->rL + (size_t)f * D : m->rR + (size_t)f * D;
        const double *ro = S[i].sgn[s] > 0 ? m->rR + (size_t)f * D : m->rL + (size_t)f * D;
        double d[3], n2 = 0.0;
        for (int a = 0; a < D; ++a) {
            d[a] = rs[a] - ro[a];          /* x_nb - x_i */
            n2 += d[a] * d[a];
        }
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) M[a * D + b] += d[a] * d[b] / n2;
    }
    double tr = 0.0;
    for (int a = 0; a < D; ++a) tr += M[a * D + a];
    if (D == 2) {
        double det = M[0] * M[3] - M[1] * M[2];
        if (!(det > 1e-12 * tr * tr)) return 0;
        Minv[0] = M[3] / det;
        Minv[1] = -M[1] / det;
        Minv[2] = -M[2] / det;
        Minv[3] = M[0] / det;
    } else {
        double c00 = M[4] * M[8] - M[5] * M[7];
        double c01 = M[5] * M[6] - M[3] * M[8];
        double c02 = M[3] * M[7] - M[4] * M[6];
        double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
        if (!(det > 1e-12 * tr * tr * tr)) return 0;
        Minv[0] = c00 / det;
        Minv[1] = (M[2] * M[7] - M[1] * M[8]) / det;
        Minv[2] = (M[1] * M[5] - M[2] * M[4]) / det;
        Minv[3] = c01 / det;
        Minv[4] = (M[0] * M[8] - M[2] * M[6]) / det;
        Minv[5] = (M[2] * M[3] - M[0] * M[5]) / det;
        Minv[6] = c02 / det;
        Minv[7] = (M[1] * M[6] - M[0] * M[7]) / det;
        Minv[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    }
    return 1;
}

/* Venkatakrishnan's limiter function, capped at 1 (R6). */
static double venkat(double d1, double d2, double eps2)
{
    double num = d1 * d1 + eps2 + 2.0 * d1 * d2;
    double den = d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2;
    double v = num / den;
    return v < 1.0 ? v : 1.0;
}

/* ---- one explicit step (Sec. 2.3, explicit reading R1/R2) --------------- */

/* Step 1 of the step: least-squares gradient (weights 1/|d|^2) of every cell,
 * array and node, and its Venkatakrishnan limiter factor L (Sec. 2.3.3, R6):
 * grad [Nc][nA][Nv][D] unlimited gradient, lim [Nc][nA][Nv] the factor, so the
 * limited gradient is lim * grad.  epsilon^2 = (K dx)^3 phi_C^2 with
 * dx = |V|^(1/D) and phi_C the cell's own value of the array at the node:
 * the (K dx)^3 of the limiter for a quantity of unit size, scaled to the size
 * of the limited value, so that the factor is the same for f and any
 * multiple of f (the distribution spans many orders of magnitude over the
 * velocity nodes).  The limiter is the least Venkatakrishnan value over the
 * cell's faces, taken with the largest (smallest) neighbour difference on
 * faces where the unlimited change grad . r is positive (negative).  A cell
 * whose LSQ matrix is singular gets a zero gradient. */
static void limited_gradients(const om_mesh *m, const om_gas *g, int Nv, const double *f_in, const slots_t *S,
                              double *grad, double *lim)
{
    const int D = m->D, nA = nArrG(g, D), Nc = m->Nc;
    double *Minv = (double *)calloc((size_t)Nc * 9, sizeof(double));
    int *lsq_ok = (int *)calloc((size_t)Nc, sizeof(int));
    double *eps2 = (double *)malloc((size_t)Nc * sizeof(double));

    for (int i = 0; i < Nc; ++i) {
        lsq_ok[i] = lsq_inverse(m, S, i, Minv + (size_t)i * 9);
        double dx = pow(m->vol[i], 1.0 / D);
        eps2[i] = pow(g->lim_K * dx, 3.0);
    }

#pragma omp parallel for schedule(static)
    for (int i = 0; i < Nc; ++i) {
        for (int a = 0; a < nA; ++a) {
            for (int k = 0; k < Nv; ++k) {
                double phi_i = f_in[((size_t)i * nA + a) * Nv + k];
                double b[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
                double dmax = 0.0, dmin = 0.0;
                for (int s = 0; s < S[i].n; ++s) {
                    int nb = slot_nb(m, S, i, s);
                    if (nb < 0) continue;
                    int f = S[i].face[s];
                    const double *rs = S[i].sgn[s] > 0 ? m->rL + (size_t)f * D : m->rR + (size_t)f * D;
                    const double *ro = S[i].sgn[s] > 0 ? m->rR + (size_t)f * D : m->rL + (size_t)f * D;
                    double d[3], n2 = 0.0;
                    for (int c = 0; c < D; ++c) {
                        d[c] = rs[c] - ro[c];
                        n2 += d[c] * d[c];
                    }
                    double dphi = f_in[((size_t)nb * nA + a) * Nv + k] - phi_i;
                    for (int c = 0; c < D; ++c) b[c] += d[c] * dphi / n2;
                    if (dphi > dmax) dmax = dphi;
                    if (dphi < dmin) dmin = dphi;
                }
                double L = 1.0;
                if (g->limiter != 0 && lsq_ok[i]) {
                    const double *Mi = Minv + (size_t)i * 9;
                    for (int r = 0; r < D; ++r)
                        for (int c = 0; c < D; ++c) gr[r] += Mi[r * D + c] * b[c];
                    if (g->limiter == 1) {
                        for (int s = 0; s < S[i].n; ++s) {
                            const double *r = slot_r(m, S, i, s);
                            double d2 = 0.0;
                            for (int c = 0; c < D; ++c) d2 += gr[c] * r[c];
                            double psi = 1.0;
                            const double e2 = eps2[i] * phi_i * phi_i;
                            if (d2 > 0.0) psi = venkat(dmax, d2, e2);
                            else if (d2 < 0.0) psi = venkat(dmin, d2, e2);
                            if (psi < L) L = psi;
                        }
                    }
                }
                size_t o = ((size_t)i * nA + a) * Nv + k;
                for (int c = 0; c < D; ++c) grad[o * D + c] = gr[c];
                lim[o] = L;
            }
        }
    }
    free(Minv); free(lsq_ok); free(eps2);
}

void om_limited_gradients(const om_mesh *m, const om_gas *g, int Nv, const double *f_in, double *grad, double *lim)
{
    slots_t *S = build_slots(m);
    limited_gradients(m, g, Nv, f_in, S, grad, lim);
    free(S);
}

double om_venkat(double d1, double d2, double eps2) { return venkat(d1, d2, eps2); }

/* Steps shared by the explicit and the implicit step: limited gradients
 * (Sec. 2.3.3), the interface distribution phi_ij of every face (Eqs. equ27,
 * equ28 with R4; boundaries R8) stored in phi [Nf][nA][Nv], and its
 * area-weighted flux moments A F_ij in F [Nf][D+2].  Returns 1 when an
 * interface state has rho <= 0 or T <= 0. */
static int interface_fluxes(const om_mesh *m, const om_gas *g, int Nv, const double *xi, const double *w,
                            double dt, const double *f_in, const slots_t *S, double *phi, double *F)
{
    const int D = m->D, nA = nArrG(g, D), NW = nWG(g, D), Nc = m->Nc, Nf = m->Nf;
    memset(F, 0, (size_t)Nf * NW * sizeof(double));
    const double h = 0.5 * dt;
    double *grad = (double *)malloc((size_t)Nc * nA * Nv * D * sizeof(double));
    double *lim = (double *)malloc((size_t)Nc * nA * Nv * sizeof(double));
    int bad = 0;

    /* 1. gradient and limiter of every cell, array and node */
    limited_gradients(m, g, Nv, f_in, S, grad, lim);

    /* 2. interface distribution and flux of every face */
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int f = 0; f < Nf; ++f) {
        const int L = m->faceL[f], R = m->faceR[f];
        const double *An = m->An + (size_t)f * D;
        double *pf = phi + (size_t)f * nA * Nv;
        /* foot value at x_f - xi h from the upwind cell (C = L if xi.n >= 0) */
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double sn = 0.0;
            for (int d = 0; d < D; ++d) sn += x[d] * An[d];
            int C;
            const double *r;
            if (sn >= 0.0) { C = L; r = m->rL + (size_t)f * D; }
            else if (R >= 0) { C = R; r = m->rR + (size_t)f * D; }
            else { for (int a = 0; a < nA; ++a) pf[a * Nv + k] = 0.0; continue; }
            for (int a = 0; a < nA; ++a) {
                size_t o = ((size_t)C * nA + a) * Nv + k;
                double dot = 0.0;
                for (int d = 0; d < D; ++d) dot += grad[o * D + d] * (r[d] - x[d] * h);
                pf[a * Nv + k] = f_in[o] + lim[o] * dot;
            }
        }
        if (R >= 0 && g->model) {
            /* Rykov interface state (R27): W from the foot values (Eq.
             * w_interface), tau from T_t; the rotational energy relaxed over
             * h toward rho R T (the second Eq. w_interface read as a backward
             * Euler step, so its factor 1 + h/(Z tau) divides); T is fixed by
             * the total energy; each heat flux relaxed over h at its rate in
             * the model (the R4 rule): lambda_t = 2/3 + (1 - omega0)/(3 Z),
             * lambda_r = 1 - (1 - delta)((1 - 1/Z) T_r/T_t + omega1/Z). */
            double Wf[6], qt[3], qr[3];
            cell_moments_rykov(D, Nv, xi, w, pf, Wf, qt, qr);
            double rho, U[3], RTt, RTr, RT;
            prim_rykov(D, Wf, &rho, U, &RTt, &RTr, &RT);
            if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) bad = 1;
            double tau = tau_of(g, rho, RTt);
            double az = h / (g->Zrot * tau);
            RTr = (Wf[D + 2] + az * rho * RT) / (1.0 + az) / rho;
            RTt = (5.0 * RT - 2.0 * RTr) / 3.0;
            double lt = 2.0 / 3.0 + (1.0 - g->omega0) / (3.0 * g->Zrot);
            double lr = 1.0 - (1.0 - g->delta) * ((1.0 - 1.0 / g->Zrot) * RTr / RTt + g->omega1 / g->Zrot);
            double qtf[3], qrf[3];
            for (int d = 0; d < D; ++d) {
                qtf[d] = tau * qt[d] / (tau + h * lt);
                qrf[d] = tau * qr[d] / (tau + h * lr);
            }
            double wa = tau / (tau + h), wb = h / (tau + h);                        /* Eq. equ28 */
            for (int k = 0; k < Nv; ++k) {
                double v[3];
                rykov(D, g, rho, U, RTt, RTr, qtf, qrf, xi + (size_t)k * D, v);
                for (int a = 0; a < nA; ++a) pf[a * Nv + k] = wa * pf[a * Nv + k] + wb * v[a];
            }
        } else if (R >= 0) {
            /* interface macroscopic state: Eq. (w_interface) */
            double Wf[5];
            cell_moments(D, Nv, xi, w, pf, Wf, NULL);
            double rho, U[3], RT, qbar[3];
            prim_of(D, Wf, &rho, U, &RT);
            {   /* heat flux of the foot distribution, Eq. (8) about U_ij */
                double qq[3] = {0, 0, 0};
                for (int k = 0; k < Nv; ++k) {
                    const double *x = xi + (size_t)k * D;
                    double c[3], c2 = 0.0;
                    for (int d = 0; d < D; ++d) { c[d] = x[d] - U[d]; c2 += c[d] * c[d]; }
                    double Hk = D == 2 ? pf[Nv + k] : 0.0;
                    for (int d = 0; d < D; ++d) qq[d] += 0.5 * w[k] * c[d] * (c2 * pf[k] + Hk);
                }
                for (int d = 0; d < D; ++d) qbar[d] = qq[d];
            }
            if (!(rho > 0.0) || !(RT > 0.0)) bad = 1;
            double tau = tau_of(g, rho, RT);
            double qf[3];
            for (int d = 0; d < D; ++d) qf[d] = tau * qbar[d] / (tau + h * g->Pr);   /* R4 */
            double wa = tau / (tau + h), wb = h / (tau + h);                        /* Eq. equ28 */
            for (int k = 0; k < Nv; ++k) {
                double gG, gH;
                shakhov(D, g->Pr, rho, U, RT, qf, xi + (size_t)k * D, &gG, &gH);
                pf[k] = wa * pf[k] + wb * gG;
                if (nA == 2) pf[Nv + k] = wa * pf[Nv + k] + wb * gH;
            }
        } else {
            /* boundary face (R8) */
            const double *B = m->bc + (size_t)(-1 - R) * 6;
            int type = (int)B[0];
            double Ub[3] = {B[2], B[3], B[4]};
            double RTb = g->R * B[5];
            double rb = B[1];
            if (type == 1) {   /* isothermal diffuse wall, zero net mass flux */
                double out = 0.0, in = 0.0;
                for (int k = 0; k < Nv; ++k) {
                    const double *x = xi + (size_t)k * D;
                    double sn = 0.0;
                    for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                    if (sn >= 0.0) out += w[k] * sn * pf[k];
                    else in += w[k] * (-sn) * maxwell(D, 1.0, Ub, RTb, x);
                }
                rb = in > 0.0 ? out / in : 0.0;
            }
            for (int k = 0; k < Nv; ++k) {
                const double *x = xi + (size_t)k * D;
                double sn = 0.0;
                for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                if (sn >= 0.0) continue;
                double gk = maxwell(D, rb, Ub, RTb, x);
                pf[k] = gk;
                if (D == 2) pf[Nv + k] = (3.0 - D) * RTb * gk;
                if (g->model) pf[(size_t)(nA - 1) * Nv + k] = RTb * gk;   /* rotational equilibrium at T_b (R29) */
            }
        }
        /* area-weighted flux  A F = sum_k w (xi . An) psi phi */
        double *Ff = F + (size_t)f * NW;
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double sn = 0.0, x2 = 0.0;
            for (int d = 0; d < D; ++d) { sn += x[d] * An[d]; x2 += x[d] * x[d]; }
            double G = pf[k], H = D == 2 ? pf[Nv + k] : 0.0;
            Ff[0] += w[k] * sn * G;
            for (int d = 0; d < D; ++d) Ff[1 + d] += w[k] * sn * x[d] * G;
            if (g->model) {
                double Rk = pf[(size_t)(nA - 1) * Nv + k];
                Ff[D + 1] += w[k] * sn * (0.5 * (x2 * G + H) + Rk);
                Ff[D + 2] += w[k] * sn * Rk;
            } else {
                Ff[D + 1] += w[k] * sn * 0.5 * (x2 * G + H);
            }
        }
    }

    free(grad); free(lim);
    return bad;
}

int om_step(const om_mesh *m, const om_gas *g, int Nv, const double *xi, const double *w,
            double dt, const double *f_in, double *f_out, double *Wc)
{
    const int D = m->D, nA = nArrG(g, D), NW = nWG(g, D), Nc = m->Nc, Nf = m->Nf;
    slots_t *S = build_slots(m);
    double *phi = (double *)malloc((size_t)Nf * nA * Nv * sizeof(double));
    double *F = (double *)calloc((size_t)Nf * NW, sizeof(double));
    int bad = interface_fluxes(m, g, Nv, xi, w, dt, f_in, S, phi, F);

    /* 3. macroscopic predictor and collision update of every cell */
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int i = 0; i < Nc; ++i) {
        double *Wi = Wc + (size_t)i * NW;
        const double *fi = f_in + (size_t)i * nA * Nv;
        double *fo = f_out + (size_t)i * nA * Nv;
        double Wt[6];
        /* explicit conservative update, R2 */
        for (int c = 0; c < NW; ++c) {
            double s = 0.0;
            for (int sl = 0; sl < S[i].n; ++sl) s += S[i].sgn[sl] * F[(size_t)S[i].face[sl] * NW + c];
            Wt[c] = Wi[c] - dt / m->vol[i] * s;
        }
        if (g->model) {
            /* Rykov (R28): the rotational source of Eq. (S_rot) taken
             * implicitly, E_rot~ = (E_rot* + a rho R T)/(1 + a), a = dt/(Z tau),
             * tau from T_t of the flux-updated state; the same tau in the
             * collision update, so the moments of f^{n+1} are W~. */
            double Wn[6], qt[3], qr[3];
            cell_moments_rykov(D, Nv, xi, w, fi, Wn, qt, qr);       /* lagged heat fluxes (R3) */
            double rho, U[3], RTt, RTr, RT;
            prim_rykov(D, Wt, &rho, U, &RTt, &RTr, &RT);
            if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) bad = 1;
            double tau = tau_of(g, rho, RTt);
            double az = dt / (g->Zrot * tau);
            Wt[D + 2] = (Wt[D + 2] + az * rho * RT) / (1.0 + az);
            prim_rykov(D, Wt, &rho, U, &RTt, &RTr, &RT);
            for (int k = 0; k < Nv; ++k) {
                const double *x = xi + (size_t)k * D;
                double v[3];
                rykov(D, g, rho, U, RTt, RTr, qt, qr, x, v);
                for (int a = 0; a < nA; ++a) {
                    double N = 0.0;
                    for (int sl = 0; sl < S[i].n; ++sl) {
                        int f = S[i].face[sl];
                        const double *An = m->An + (size_t)f * D;
                        double sn = 0.0;
                        for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                        N += S[i].sgn[sl] * sn * phi[((size_t)f * nA + a) * Nv + k];
                    }
                    fo[a * Nv + k] = (fi[a * Nv + k] / dt + v[a] / tau - N / m->vol[i]) / (1.0 / dt + 1.0 / tau);
                }
            }
            for (int c = 0; c < NW; ++c) Wi[c] = Wt[c];
            continue;
        }
        /* lagged heat flux of f^n (R3) */
        double Wn[5], qn[3];
        cell_moments(D, Nv, xi, w, fi, Wn, qn);
        double rho, U[3], RT;
        prim_of(D, Wt, &rho, U, &RT);
        if (!(rho > 0.0) || !(RT > 0.0)) bad = 1;
        double tau = tau_of(g, rho, RT);
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double gG, gH;
            shakhov(D, g->Pr, rho, U, RT, qn, x, &gG, &gH);
            for (int a = 0; a < nA; ++a) {
                double N = 0.0;
                for (int sl = 0; sl < S[i].n; ++sl) {
                    int f = S[i].face[sl];
                    const double *An = m->An + (size_t)f * D;
                    double sn = 0.0;
                    for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                    N += S[i].sgn[sl] * sn * phi[((size_t)f * nA + a) * Nv + k];
                }
                double ge = a == 0 ? gG : gH;
                /* diagonal of Eq. (SGS_phi): explicit transport, implicit collision (R1) */
                fo[a * Nv + k] = (fi[a * Nv + k] / dt + ge / tau - N / m->vol[i]) / (1.0 / dt + 1.0 / tau);
            }
        }
        for (int c = 0; c < NW; ++c) Wi[c] = Wt[c];
    }

    free(S); free(phi); free(F);
    return bad ? -5 : 0;
}

/* ---- implicit step (IUGKS, Sec. 2.3.1 macroscopic and microscopic) ---- */

/* Greedy colouring of the cells in index order (each cell takes the smallest
 * colour none of its face neighbours has): cells of one colour share no face,
 * so a colour-by-colour Gauss-Seidel sweep is a sweep in the cell order
 * "colour 0 cells ascending, colour 1 cells ascending, ...".  Returns the
 * number of colours. */
int om_colors(const om_mesh *m, int *color)
{
    slots_t *S = build_slots(m);
    int nc = 0;
    for (int i = 0; i < m->Nc; ++i) color[i] = -1;
    for (int i = 0; i < m->Nc; ++i) {
        unsigned used = 0;
        for (int s = 0; s < S[i].n; ++s) {
            int j = slot_nb(m, S, i, s);
            if (j >= 0 && color[j] >= 0) used |= 1u << color[j];
        }
        int c = 0;
        while (used & (1u << c)) ++c;
        color[i] = c;
        if (c + 1 > nc) nc = c + 1;
    }
    free(S);
    return nc;
}

/* Euler flux of W through the unit normal n: (rho U.n, rho U (U.n) + p n,
 * (rho E + p) U.n), p = rho R T (monatomic). */
static void euler_flux(int D, const double *W, const double *n, double *G)
{
    double rho, U[3], RT;
    prim_of(D, W, &rho, U, &RT);
    double un = 0.0;
    for (int d = 0; d < D; ++d) un += U[d] * n[d];
    double p = rho * RT;
    G[0] = rho * un;
    for (int d = 0; d < D; ++d) G[1 + d] = W[1 + d] * un + p * n[d];
    G[D + 1] = (W[D + 1] + p) * un;
}

/* Euler flux of a diatomic gas (Rykov W): p = rho R T with the equilibrium
 * temperature of the total energy; rho E_rot is carried with the flow (R31). */
static void euler_flux_rykov(int D, const double *W, const double *n, double *G)
{
    double rho, U[3], RTt, RTr, RT;
    prim_rykov(D, W, &rho, U, &RTt, &RTr, &RT);
    double un = 0.0;
    for (int d = 0; d < D; ++d) un += U[d] * n[d];
    double p = rho * RT;
    G[0] = rho * un;
    for (int d = 0; d < D; ++d) G[1 + d] = W[1 + d] * un + p * n[d];
    G[D + 1] = (W[D + 1] + p) * un;
    G[D + 2] = W[D + 2] * un;
}

static void euler_flux_g(const om_gas *g, int D, const double *W, const double *n, double *G)
{
    if (g->model) euler_flux_rykov(D, W, n, G);
    else euler_flux(D, W, n, G);
}

/* Spectral radius of the Roe-type dissipation at a face (Eq. after Eq. Roe):
 * r = |U.n| + a + 2 mu / (rho dl), from the mean of the primitive states of
 * the two sides (reading: the paper leaves the interface state open), a the
 * sound speed sqrt(5/3 R T) of a monatomic gas, mu the VHS viscosity. */
static double roe_radius(const om_gas *g, int D, const double *WL, const double *WR, const double *n, double dl)
{
    double rl, Ul[3], RTl, rr, Ur[3], RTr;
    if (g->model) {
        /* Rykov (R31): a = sqrt(7/5 R T) with the equilibrium T, mu at the mean T_t */
        double tl, ql, tr, qr;
        prim_rykov(D, WL, &rl, Ul, &tl, &ql, &RTl);
        prim_rykov(D, WR, &rr, Ur, &tr, &qr, &RTr);
        double rho = 0.5 * (rl + rr), RT = 0.5 * (RTl + RTr), RTt = 0.5 * (tl + tr), un = 0.0;
        for (int d = 0; d < D; ++d) un += 0.5 * (Ul[d] + Ur[d]) * n[d];
        double mu = g->mu_ref * pow(RTt / g->R / g->T_ref, g->omega);
        return fabs(un) + sqrt(7.0 / 5.0 * RT) + 2.0 * mu / (rho * dl);
    }
    prim_of(D, WL, &rl, Ul, &RTl);
    prim_of(D, WR, &rr, Ur, &RTr);
    double rho = 0.5 * (rl + rr), RT = 0.5 * (RTl + RTr), un = 0.0;
    for (int d = 0; d < D; ++d) un += 0.5 * (Ul[d] + Ur[d]) * n[d];
    double T = RT / g->R;
    double mu = g->mu_ref * pow(T / g->T_ref, g->omega);
    return fabs(un) + sqrt(5.0 / 3.0 * RT) + 2.0 * mu / (rho * dl);
}

/* One implicit step: the interface distribution and fluxes at t^n as in the
 * explicit step, then
 *  - macroscopic: Eq. (SGS_w) for dW = W~ - W^n, solved by k_macro symmetric
 *    Gauss-Seidel iterations (a forward and a backward sweep over the colours
 *    each); boundary faces enter the diagonal with their radius and a fixed
 *    ghost state (no off-diagonal term);
 *  - microscopic: Eq. (SGS_phi) for dphi = phi^{n+1} - phi^n with tau~, g~
 *    from W~ and the lagged heat flux of f^n (R3), k_micro symmetric sweeps;
 *    boundary faces bring no dphi of a neighbour.
 * f_out = f_in + dphi, Wc <- W~.  color: a proper colouring (om_colors).
 * Returns -5 when a state has rho <= 0 or T <= 0. */
int om_step_implicit(const om_mesh *m, const om_gas *g, int Nv, const double *xi, const double *w,
                     double dt, const double *f_in, double *f_out, double *Wc,
                     const int *color, int ncolor, int k_macro, int k_micro)
{
    const int D = m->D, nA = nArrG(g, D), NW = nWG(g, D), Nc = m->Nc, Nf = m->Nf;
    slots_t *S = build_slots(m);
    double *phi = (double *)malloc((size_t)Nf * nA * Nv * sizeof(double));
    double *F = (double *)calloc((size_t)Nf * NW, sizeof(double));
    int bad = interface_fluxes(m, g, Nv, xi, w, dt, f_in, S, phi, F);

    /* cells in sweep order: by colour, ascending index within a colour */
    int *order = (int *)malloc((size_t)Nc * sizeof(int));
    int *cstart = (int *)calloc((size_t)ncolor + 1, sizeof(int));
    for (int i = 0; i < Nc; ++i) cstart[color[i] + 1]++;
    for (int c = 0; c < ncolor; ++c) cstart[c + 1] += cstart[c];
    {
        int *pos = (int *)malloc((size_t)ncolor * sizeof(int));
        for (int c = 0; c < ncolor; ++c) pos[c] = cstart[c];
        for (int i = 0; i < Nc; ++i) order[pos[color[i]]++] = i;
        free(pos);
    }

    /* ---- macroscopic system, Eq. (SGS_w) */
    double *rad = (double *)malloc((size_t)Nf * sizeof(double));      /* A r per face */
    for (int f = 0; f < Nf; ++f) {
        const int L = m->faceL[f], R = m->faceR[f];
        const double *An = m->An + (size_t)f * D;
        double A = 0.0, n[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) A += An[d] * An[d];
        A = sqrt(A);
        for (int d = 0; d < D; ++d) n[d] = An[d] / A;
        double dl = 0.0;
        if (R >= 0) {
            for (int d = 0; d < D; ++d) {
                double e = m->rL[(size_t)f * D + d] - m->rR[(size_t)f * D + d];
                dl += e * e;
            }
        } else {
            for (int d = 0; d < D; ++d) dl += 4.0 * m->rL[(size_t)f * D + d] * m->rL[(size_t)f * D + d];
        }
        dl = sqrt(dl);
        const double *WR = R >= 0 ? Wc + (size_t)R * NW : Wc + (size_t)L * NW;
        rad[f] = A * roe_radius(g, D, Wc + (size_t)L * NW, WR, n, dl);
    }
    double *dW = (double *)calloc((size_t)Nc * NW, sizeof(double));
    double *Wt = (double *)malloc((size_t)Nc * NW * sizeof(double));
    memcpy(Wt, Wc, (size_t)Nc * NW * sizeof(double));
    for (int it = 0; it < k_macro; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int q = 0; q < Nc; ++q) {
                const int i = order[dir == 0 ? q : Nc - 1 - q];
                double diag = m->vol[i] / dt, rhs[6];
                for (int c = 0; c < NW; ++c) {
                    double acc = 0.0;
                    for (int sl = 0; sl < S[i].n; ++sl) acc += S[i].sgn[sl] * F[(size_t)S[i].face[sl] * NW + c];
                    rhs[c] = -acc;
                }
                for (int sl = 0; sl < S[i].n; ++sl) {
                    const int f = S[i].face[sl];
                    diag += 0.5 * rad[f];
                    const int j = slot_nb(m, S, i, sl);
                    if (j < 0) continue;
                    const double *An = m->An + (size_t)f * D;
                    double A = 0.0, n[3] = {0, 0, 0};
                    for (int d = 0; d < D; ++d) A += An[d] * An[d];
                    A = sqrt(A);
                    for (int d = 0; d < D; ++d) n[d] = S[i].sgn[sl] * An[d] / A;
                    double Gt[6], Gn[6];
                    euler_flux_g(g, D, Wt + (size_t)j * NW, n, Gt);
                    euler_flux_g(g, D, Wc + (size_t)j * NW, n, Gn);
                    for (int c = 0; c < NW; ++c)
                        rhs[c] += -0.5 * A * (Gt[c] - Gn[c]) + 0.5 * rad[f] * dW[(size_t)j * NW + c];
                }
                double diag_rot = diag;
                if (g->model) {
                    /* rotational source of Eq. (SGS_wrot), (rho R T - rho E_rot^n)/(Z tau), with
                     * rho R T and tau from the cell's current W~ (reading R32); its implicit
                     * part V/(Z tau) joins the diagonal of the rho E_rot row */
                    double rho, U[3], RTt, RTr, RT;
                    prim_rykov(D, Wt + (size_t)i * NW, &rho, U, &RTt, &RTr, &RT);
                    if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) bad = 1;
                    double tau = tau_of(g, rho, RTt), V = m->vol[i];
                    rhs[D + 2] += V * (rho * RT - Wc[(size_t)i * NW + D + 2]) / (g->Zrot * tau);
                    diag_rot = diag + V / (g->Zrot * tau);
                }
                for (int c = 0; c < NW; ++c) {
                    dW[(size_t)i * NW + c] = rhs[c] / (c == D + 2 ? diag_rot : diag);
                    Wt[(size_t)i * NW + c] = Wc[(size_t)i * NW + c] + dW[(size_t)i * NW + c];
                }
            }
        }
    }

    /* ---- microscopic system, Eq. (SGS_phi), every node and array */
    double *res = (double *)malloc((size_t)Nc * nA * Nv * sizeof(double));
    double *dg = (double *)malloc((size_t)Nc * Nv * sizeof(double));       /* diagonal per cell and node */
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int i = 0; i < Nc; ++i) {
        const double *fi = f_in + (size_t)i * nA * Nv;
        if (g->model) {
            /* Rykov: g~ from W~ with the lagged q_t, q_r of f^n, tau~ from T_t of W~ */
            double Wr[6], qt[3], qr[3];
            cell_moments_rykov(D, Nv, xi, w, fi, Wr, qt, qr);
            double rho, U[3], RTt, RTr, RT;
            prim_rykov(D, Wt + (size_t)i * NW, &rho, U, &RTt, &RTr, &RT);
            if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) bad = 1;
            double tau = tau_of(g, rho, RTt), V = m->vol[i];
            for (int k = 0; k < Nv; ++k) {
                const double *x = xi + (size_t)k * D;
                double v[3], out = 0.0;
                rykov(D, g, rho, U, RTt, RTr, qt, qr, x, v);
                for (int sl = 0; sl < S[i].n; ++sl) {
                    const double *An = m->An + (size_t)S[i].face[sl] * D;
                    double sn = 0.0;
                    for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                    sn *= S[i].sgn[sl];
                    if (sn >= 0.0) out += sn;
                }
                dg[(size_t)i * Nv + k] = V / dt + V / tau + out;
                for (int a = 0; a < nA; ++a) {
                    double N = 0.0;
                    for (int sl = 0; sl < S[i].n; ++sl) {
                        int f = S[i].face[sl];
                        const double *An = m->An + (size_t)f * D;
                        double sn = 0.0;
                        for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                        N += S[i].sgn[sl] * sn * phi[((size_t)f * nA + a) * Nv + k];
                    }
                    res[((size_t)i * nA + a) * Nv + k] = V * (v[a] - fi[a * Nv + k]) / tau - N;
                }
            }
            continue;
        }
        double Wn[5], qn[3];
        cell_moments(D, Nv, xi, w, fi, Wn, qn);          /* lagged heat flux of f^n (R3) */
        double rho, U[3], RT;
        prim_of(D, Wt + (size_t)i * NW, &rho, U, &RT);
        if (!(rho > 0.0) || !(RT > 0.0)) bad = 1;
        double tau = tau_of(g, rho, RT), V = m->vol[i];
        for (int k = 0; k < Nv; ++k) {
            const double *x = xi + (size_t)k * D;
            double gG, gH, out = 0.0;
            shakhov(D, g->Pr, rho, U, RT, qn, x, &gG, &gH);
            for (int sl = 0; sl < S[i].n; ++sl) {
                const double *An = m->An + (size_t)S[i].face[sl] * D;
                double sn = 0.0;
                for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                sn *= S[i].sgn[sl];
                if (sn >= 0.0) out += sn;
            }
            dg[(size_t)i * Nv + k] = V / dt + V / tau + out;
            for (int a = 0; a < nA; ++a) {
                double N = 0.0;
                for (int sl = 0; sl < S[i].n; ++sl) {
                    int f = S[i].face[sl];
                    const double *An = m->An + (size_t)f * D;
                    double sn = 0.0;
                    for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                    N += S[i].sgn[sl] * sn * phi[((size_t)f * nA + a) * Nv + k];
                }
                double ge = a == 0 ? gG : gH;
                res[((size_t)i * nA + a) * Nv + k] = V * (ge - fi[a * Nv + k]) / tau - N;
            }
        }
    }
    double *dphi = (double *)calloc((size_t)Nc * nA * Nv, sizeof(double));
    for (int it = 0; it < k_micro; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int q = 0; q < Nc; ++q) {
                const int i = order[dir == 0 ? q : Nc - 1 - q];
                for (int k = 0; k < Nv; ++k) {
                    const double *x = xi + (size_t)k * D;
                    for (int a = 0; a < nA; ++a) {
                        double acc = res[((size_t)i * nA + a) * Nv + k];
                        for (int sl = 0; sl < S[i].n; ++sl) {
                            const int j = slot_nb(m, S, i, sl);
                            if (j < 0) continue;
                            const double *An = m->An + (size_t)S[i].face[sl] * D;
                            double sn = 0.0;
                            for (int d = 0; d < D; ++d) sn += x[d] * An[d];
                            sn *= S[i].sgn[sl];
                            if (sn < 0.0) acc -= sn * dphi[((size_t)j * nA + a) * Nv + k];
                        }
                        dphi[((size_t)i * nA + a) * Nv + k] = acc / dg[(size_t)i * Nv + k];
                    }
                }
            }
        }
    }
    for (size_t e = 0; e < (size_t)Nc * nA * Nv; ++e) f_out[e] = f_in[e] + dphi[e];
    memcpy(Wc, Wt, (size_t)Nc * NW * sizeof(double));

    free(S); free(phi); free(F); free(order); free(cstart); free(rad); free(dW); free(Wt);
    free(res); free(dg); free(dphi);
    return bad ? -5 : 0;
}

/* ---- adaptive criterion (Sec. 3.4) ------------------------------------- */

/* M_k = max over cells of max(M1, M2) (Eqs. criterion_rho/_e/_mk), with the
 * cell's rho, U and internal energy from the given conserved W.  The
 * operation order is fixed: wg = w G; M1 = wg / rho;
 * c2 = sum_d (xi_d - U_d)^2 left to right; M2 = ((0.5 wg) c2) / e_int,
 * e_int = rho E - 0.5 (sum_d m_d m_d) / rho.  M2 uses G only (R9). */
void om_criterion(int D, int Nc, int Nv, const double *xi, const double *w, const double *f,
                  const double *Wc, double *M)
{
    om_criterion_nw(D, nArr(D), D + 2, Nc, Nv, xi, w, f, Wc, M);
}

/* The same with nA arrays per cell and nw conserved variables per cell (the
 * Rykov model: e_int includes the rotational energy, R30). */
void om_criterion_nw(int D, int nA, int nw, int Nc, int Nv, const double *xi, const double *w,
                     const double *f, const double *Wc, double *M)
{
    for (int k = 0; k < Nv; ++k) M[k] = -INFINITY;
    for (int i = 0; i < Nc; ++i) {
        const double *W = Wc + (size_t)i * nw;
        double rho = W[0];
        double U[3], mm = 0.0;
        for (int d = 0; d < D; ++d) {
            U[d] = W[1 + d] / rho;
            mm = mm + W[1 + d] * W[1 + d];
        }
        double eint = W[D + 1] - 0.5 * mm / rho;
        const double *G = f + (size_t)i * nA * Nv;
        for (int k = 0; k < Nv; ++k) {
            double wg = w[k] * G[k];
            double m1 = wg / rho;
            double c2 = 0.0;
            for (int d = 0; d < D; ++d) {
                double c = xi[(size_t)k * D + d] - U[d];
                c2 = c2 + c * c;
            }
            double m2 = ((0.5 * wg) * c2) / eint;
            double mk = m1 > m2 ? m1 : m2;
            if (mk > M[k]) M[k] = mk;
        }
    }
}

/* ---- marks and the new tree (Sec. 3.1, 3.4; readings R10, R11, R14) ---- */
/* Split a leaf when s*M_k > C1 and its level < its cap: lcap[k] when
 * lcap is given (the refinement zones of Sec. 3.5), else max_refine.  Merge 2^D
 * sibling leaves into their parent when all of them satisfy s*M < C2 (their
 * level >= 1).  New order is depth first: a kept leaf emits itself, a split
 * leaf its children in digit order, a merged group its parent.  src/kind
 * give, per new node, the old node it copies or the first of the 2^D old
 * siblings it averages.  Returns the new count, or -1 if it exceeds cap. */
int om_adapt_tree(int D, int Nv, const int *level, const int *base, const unsigned *key,
                  const double *M, double s, double C1, double C2, int max_refine, const int *lcap, int cap,
                  int *nlevel, int *nbase, unsigned *nkey, int *src, int *kind)
{
    const int nch = 1 << D;
    int n = 0;
    int k = 0;
    while (k < Nv) {
        int group = 0;
        if (level[k] >= 1 && (key[k] & (unsigned)(nch - 1)) == 0u && k + nch <= Nv) {
            group = 1;
            for (int c = 0; c < nch; ++c) {
                int kk = k + c;
                if (level[kk] != level[k] || base[kk] != base[k] || key[kk] != key[k] + (unsigned)c ||
                    !(s * M[kk] < C2))
                    group = 0;
            }
        }
        if (group) {
            if (n + 1 > cap) return -1;
            nlevel[n] = level[k] - 1;
            nbase[n] = base[k];
            nkey[n] = key[k] >> D;
            src[n] = k;
            kind[n] = OM_MERGE;
            n++;
            k += nch;
            continue;
        }
        if (s * M[k] > C1 && level[k] < (lcap ? lcap[k] : max_refine)) {
            if (n + nch > cap) return -1;
            for (int c = 0; c < nch; ++c) {
                nlevel[n] = level[k] + 1;
                nbase[n] = base[k];
                nkey[n] = (key[k] << D) | (unsigned)c;
                src[n] = k;
                kind[n] = OM_COPY;
                n++;
            }
        } else {
            if (n + 1 > cap) return -1;
            nlevel[n] = level[k];
            nbase[n] = base[k];
            nkey[n] = key[k];
            src[n] = k;
            kind[n] = OM_COPY;
            n++;
        }
        k++;
    }
    return n;
}

/* Consanguinity reconstruction (Sec. 3.2): a child copies its parent, a
 * merged parent takes the mean of its children, summed pairwise
 * ((c0 + c1) + (c2 + c3)) / 4 in 2D and the three-level pairwise sum / 8 in 3D. */
void om_remap(int D, int Nc, int Nv_old, const double *f_old, int Nv_new,
              const int *src, const int *kind, double *f_new)
{
    om_remap_n(D, nArr(D), Nc, Nv_old, f_old, Nv_new, src, kind, f_new);
}

void om_remap_n(int D, int nA, int Nc, int Nv_old, const double *f_old, int Nv_new,
                const int *src, const int *kind, double *f_new)
{
    for (int i = 0; i < Nc; ++i) {
        for (int a = 0; a < nA; ++a) {
            const double *fo = f_old + ((size_t)i * nA + a) * Nv_old;
            double *fn = f_new + ((size_t)i * nA + a) * Nv_new;
            for (int k = 0; k < Nv_new; ++k) {
                const double *c = fo + src[k];
                if (kind[k] == OM_COPY) fn[k] = c[0];
                else if (D == 2) fn[k] = ((c[0] + c[1]) + (c[2] + c[3])) * 0.25;
                else fn[k] = (((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]))) * 0.125;
            }
        }
    }
}

/* Conservation correction (Sec. 3.3): f = f' + g^eq(W) - g^eq(W'), with
 * W' the discrete moments of f'; repeated `iters` times (R12).  Returns the
 * largest remaining relative gap |M[f] - W| over cells and components
 * (density relative to rho, momentum to rho sqrt(2 R T) + |rho U|, energy
 * relative to rho E). */
double om_correct(int D, int Nc, int Nv, const double *xi, const double *w, double R,
                  int iters, const double *Wc_target, double *f)
{
    int nA = nArr(D);
    double worst = 0.0;
    (void)R;
    for (int i = 0; i < Nc; ++i) {
        const double *Wt = Wc_target + (size_t)i * (D + 2);
        double *fi = f + (size_t)i * nA * Nv;
        double rho, U[3], RT;
        prim_of(D, Wt, &rho, U, &RT);
        for (int it = 0; it < iters; ++it) {
            double Wp[5];
            cell_moments(D, Nv, xi, w, fi, Wp, NULL);
            double rp, Up[3], RTp;
            prim_of(D, Wp, &rp, Up, &RTp);
            for (int k = 0; k < Nv; ++k) {
                const double *x = xi + (size_t)k * D;
                double ga = maxwell(D, rho, U, RT, x);
                double gb = maxwell(D, rp, Up, RTp, x);
                fi[k] += ga - gb;
                if (nA == 2) fi[Nv + k] += (3.0 - D) * (RT * ga - RTp * gb);
            }
        }
        double Wp[5];
        cell_moments(D, Nv, xi, w, fi, Wp, NULL);
        double mref = 0.0;
        for (int d = 0; d < D; ++d) mref += Wt[1 + d] * Wt[1 + d];
        mref = sqrt(mref) + rho * sqrt(2.0 * RT);
        double e = fabs(Wp[0] - Wt[0]) / fabs(Wt[0]);
        for (int d = 0; d < D; ++d) {
            double t = fabs(Wp[1 + d] - Wt[1 + d]) / mref;
            if (t > e) e = t;
        }
        double t = fabs(Wp[D + 1] - Wt[D + 1]) / fabs(Wt[D + 1]);
        if (t > e) e = t;
        if (e > worst || e != e) worst = e;
    }
    return worst;
}

/* Conservation correction for the Rykov model (Sec. 3.3 with R30): the
 * equilibrium set g^M(W) = (G = g^eq(rho, U, T_t), H = (3 - D) R T_t G,
 * R = R T_r G) carries (rho, rho U, rho E, rho E_rot) of W, and
 * f <- f + g^M(W) - g^M(W') with W' the moments of f, `iters` times.
 * Returns the largest relative gap as om_correct, with rho E_rot relative to
 * rho E. */
double om_correct_rykov(int D, int Nc, int Nv, const double *xi, const double *w, double R,
                        int iters, const double *Wc_target, double *f)
{
    const int nA = D == 2 ? 3 : 2, NW = D + 3;
    double worst = 0.0;
    (void)R;
    for (int i = 0; i < Nc; ++i) {
        const double *Wt = Wc_target + (size_t)i * NW;
        double *fi = f + (size_t)i * nA * Nv;
        double rho, U[3], RTt, RTr, RT;
        prim_rykov(D, Wt, &rho, U, &RTt, &RTr, &RT);
        for (int it = 0; it < iters; ++it) {
            double Wp[6];
            cell_moments_rykov(D, Nv, xi, w, fi, Wp, NULL, NULL);
            double rp, Up[3], RTtp, RTrp, RTp;
            prim_rykov(D, Wp, &rp, Up, &RTtp, &RTrp, &RTp);
            for (int k = 0; k < Nv; ++k) {
                const double *x = xi + (size_t)k * D;
                double ga = maxwell(D, rho, U, RTt, x);
                double gb = maxwell(D, rp, Up, RTtp, x);
                fi[k] += ga - gb;
                if (D == 2) fi[Nv + k] += (3.0 - D) * (RTt * ga - RTtp * gb);
                fi[(size_t)(nA - 1) * Nv + k] += RTr * ga - RTrp * gb;
            }
        }
        double Wp[6];
        cell_moments_rykov(D, Nv, xi, w, fi, Wp, NULL, NULL);
        double mref = 0.0;
        for (int d = 0; d < D; ++d) mref += Wt[1 + d] * Wt[1 + d];
        mref = sqrt(mref) + rho * sqrt(2.0 * RT);
        double e = fabs(Wp[0] - Wt[0]) / fabs(Wt[0]);
        for (int d = 0; d < D; ++d) {
            double t = fabs(Wp[1 + d] - Wt[1 + d]) / mref;
            if (t > e) e = t;
        }
        for (int c = D + 1; c < NW; ++c) {
            double t = fabs(Wp[c] - Wt[c]) / fabs(Wt[D + 1]);
            if (t > e) e = t;
        }
        if (e > worst || e != e) worst = e;
    }
    return worst;
}
