// Rykov model (diatomic gas, K = 2 rotational degrees of freedom) on the GPU:
// the explicit UGKS step, the cell moments and the conservation correction
// for the reduced distributions G, H, R in 2D and G, R in 3D (Sec. 2.1,
// Eqs. updat_W, 8, GHR_equ, 11-13; interface state of Sec. 2.3.3).
//
// W = (rho, rho U, rho E, rho E_rot): rho E = int (xi^2 G + H)/2 + R,
// rho E_rot = int R = rho R T_r, (3/2) rho R T_t = rho E - rho U^2/2 - rho E_rot,
// and the equilibrium temperature T = (3 T_t + 2 T_r) / 5.
//
// The kernels take one block per face or cell.  The FP64 form sums over the
// nodes in FP64 directly; the FP32 (mixed) form sums raw moments in FP32 per
// thread and in FP64 across warps.  The equilibrium is evaluated in the
// element type.
#include <algorithm>

#include "avs_dev.cuh"
#include "avs_internal.h"

namespace avs {
namespace {

constexpr int RK_NT = 128;

template <int D>
struct RkNA {
    static constexpr int v = D == 2 ? 3 : 2;
};

// gas constants and the Rykov coefficients: Z_rot, iz = 1/Z_rot, omega0, omega1, delta
struct RkGas {
    double R, mu_ref, T_ref, omega, Z, iz, om0, om1, dl;
};

// conserved -> rho, U, R T_t, R T_r, R T
template <int D>
__device__ void rk_prim(const double* W, double& rho, double* U, double& RTt, double& RTr, double& RT)
{
    rho = W[0];
    double m2 = 0.0;
    for (int d = 0; d < 3; ++d) U[d] = 0.0;
    for (int d = 0; d < D; ++d) {
        U[d] = W[1 + d] / rho;
        m2 += W[1 + d] * W[1 + d];
    }
    RTr = W[D + 2] / rho;
    RTt = (W[D + 1] - 0.5 * m2 / rho - W[D + 2]) / (1.5 * rho);
    RT = (W[D + 1] - 0.5 * m2 / rho) / (2.5 * rho);
}

// tau = mu(T_t) / p_t with the VHS viscosity (Eq. 3)
__device__ double rk_tau(const RkGas& g, double rho, double RTt)
{
    const double T = RTt / g.R;
    const double mu = g.mu_ref * pow(T / g.T_ref, g.omega);
    return mu / (rho * RTt);
}

// Parameters of the Rykov equilibrium of one state, in the element type.
template <typename T>
struct RkEq {
    T U[3];
    T pt, pr;                 // rho / (2 pi R T_t)^(D/2), rho / (2 pi R T)^(D/2)
    T RTt, RTr, RT;
    T iRTt, iRT;              // 1 / R T_t, 1 / R T (the FP32 form multiplies by them)
    T at[3], ar[3];           // q_t / (15 p_t R T_t), omega0 q_t / (15 p R T)
    T bt[3], br[3];           // (1 - delta) q_r / (p_t R T_t), omega1 (1 - delta) q_r / (p R T)
    T iz;
};

template <int D, typename T>
__device__ RkEq<T> rk_make(const RkGas& g, double rho, const double* U, double RTt, double RTr, const double* qt,
                           const double* qr)
{
    RkEq<T> e;
    const double RT = (3.0 * RTt + 2.0 * RTr) / 5.0;
    const double pt = rho * RTt, p = rho * RT;
    for (int d = 0; d < 3; ++d) {
        const bool on = d < D;
        e.U[d] = on ? (T)U[d] : T(0);
        e.at[d] = on ? (T)(qt[d] / (15.0 * pt * RTt)) : T(0);
        e.ar[d] = on ? (T)(g.om0 * qt[d] / (15.0 * p * RT)) : T(0);
        e.bt[d] = on ? (T)((1.0 - g.dl) * qr[d] / (pt * RTt)) : T(0);
        e.br[d] = on ? (T)(g.om1 * (1.0 - g.dl) * qr[d] / (p * RT)) : T(0);
    }
    e.pt = (T)(rho / pow(2.0 * AVS_PI * RTt, 0.5 * D));
    e.pr = (T)(rho / pow(2.0 * AVS_PI * RT, 0.5 * D));
    e.RTt = (T)RTt;
    e.RTr = (T)RTr;
    e.RT = (T)RT;
    e.iRTt = (T)(1.0 / RTt);
    e.iRT = (T)(1.0 / RT);
    e.iz = (T)g.iz;
    return e;
}

// Eqs. (GHR_equ), (11)-(13) at one node: out[0] = g^G, out[1] = g^H (2D),
// out[NA - 1] = g^R.
template <int D, typename T>
__device__ __forceinline__ void rk_eval(const RkEq<T>& e, const T* x, T* out)
{
    T c2 = T(0), cat = T(0), car = T(0), cbt = T(0), cbr = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const T c = x[d] - e.U[d];
        c2 += c * c;
        cat += c * e.at[d];
        car += c * e.ar[d];
        cbt += c * e.bt[d];
        cbr += c * e.br[d];
    }
    // c^2 / R T: divisions in the FP64 form (as the oracle), reciprocals in FP32
    T st, sr;
    if constexpr (sizeof(T) == 4) {
        st = c2 * e.iRTt;
        sr = c2 * e.iRT;
    } else {
        st = c2 / e.RTt;
        sr = c2 / e.RT;
    }
    const T gt = e.pt * ex(sizeof(T) == 4 ? T(-0.5) * st : -c2 / (T(2) * e.RTt));
    const T gr = e.pr * ex(sizeof(T) == 4 ? T(-0.5) * sr : -c2 / (T(2) * e.RT));
    const T Gt = gt * (T(1) + cat * (st - T(D + 2)));
    const T Gr = gr * (T(1) + car * (sr - T(D + 2)));
    const T a = T(1) - e.iz;
    out[0] = a * Gt + e.iz * Gr;
    if (D == 2) {
        const T Ht = e.RTt * gt * (T(1) + cat * (st - T(D)));
        const T Hr = e.RT * gr * (T(1) + car * (sr - T(D)));
        out[1] = a * Ht + e.iz * Hr;
    }
    const T Rt = e.RTr * (Gt + cbt * gt);
    const T Rr = e.RT * (Gr + cbr * gr);
    out[RkNA<D>::v - 1] = a * Rt + e.iz * Rr;
}

// Moments of one cell's f (all threads of the block): W = (rho, rho U, rho E,
// rho E_rot) and, when qt is given, q_t = int c (c^2 G + H)/2 and q_r = int c R
// about the cell's mean velocity (Eqs. updat_W, 8).  FP64 sums.
template <int D, typename T>
__device__ void rk_cell_mom(const T* fi, int Nv, int Nvp, const double* __restrict__ xi,
                            const double* __restrict__ w, double* W, double* qt, double* qr, double* sred,
                            double* sout)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3;
    double acc[NW];
#pragma unroll
    for (int m = 0; m < NW; ++m) acc[m] = 0.0;
    for (int k = threadIdx.x; k < Nv; k += RK_NT) {
        const double wk = w[k];
        double x[D], x2 = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            x[d] = xi[(size_t)k * D + d];
            x2 += x[d] * x[d];
        }
        const double G = (double)fi[k], H = D == 2 ? (double)fi[Nvp + k] : 0.0;
        const double Rr = (double)fi[(size_t)(NA - 1) * Nvp + k];
        acc[0] += wk * G;
#pragma unroll
        for (int d = 0; d < D; ++d) acc[1 + d] += wk * x[d] * G;
        acc[D + 1] += wk * (0.5 * (x2 * G + H) + Rr);
        acc[D + 2] += wk * Rr;
    }
    block_sum<NW, RK_NT>(acc, sred, sout);
#pragma unroll
    for (int m = 0; m < NW; ++m) W[m] = sout[m];
    if (!qt) return;
    double U[D], a[2 * D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        U[d] = W[1 + d] / W[0];
        a[d] = a[D + d] = 0.0;
    }
    for (int k = threadIdx.x; k < Nv; k += RK_NT) {
        const double wk = w[k];
        double c[D], c2 = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            c[d] = xi[(size_t)k * D + d] - U[d];
            c2 += c[d] * c[d];
        }
        const double G = (double)fi[k], H = D == 2 ? (double)fi[Nvp + k] : 0.0;
        const double Rr = (double)fi[(size_t)(NA - 1) * Nvp + k];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            a[d] += 0.5 * wk * c[d] * (c2 * G + H);
            a[D + d] += wk * c[d] * Rr;
        }
    }
    block_sum<2 * D, RK_NT>(a, sred, sout);
    for (int d = 0; d < D; ++d) {
        qt[d] = sout[d];
        qr[d] = sout[D + d];
    }
}

template <typename T>
struct RkP {
    int Nv, Nvp, Nc, limiter;
    double dt, h;
    RkGas g;
    const int* order;         // face processing order (by lower cell index: neighbouring faces share L2 rows)
    const int* faceL;
    const int* faceR;
    const double* An;
    const double* rL;
    const double* rR;
    const double* bc;
    const double* xi;
    const double* w;
    const double* vol;
    const int* slot;
    const unsigned char* nslot;
    const T* f;               // f^n [cell][NA][Nvp]
    const T* G;               // limited gradients [cell][NA][D][Nvp], or null (first order)
    T* FX;                    // [face][NA][Nvp]: foot values, then the face flux (xi . A n) phi
    double* AF;               // [face][D + 3] area-weighted flux of W
    const double* Win;
    double* Wout;
    T* fout;
    int* err;
};

// One face: foot values from the upwind cell, the Rykov interface state
// (reading R27) and phi_ij = tau/(tau+h) phi_bar + h/(tau+h) g (Eq. equ28);
// boundary faces as in R8/R29.  Writes the per-node face flux and A F.
template <int D, typename T>
__global__ void __launch_bounds__(RK_NT) rk_face(RkP<T> P)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3;
    __shared__ double sred[(RK_NT / 32) * 6], sout[6];
    __shared__ RkEq<T> eq;
    __shared__ double blend[2];
    const int f = P.order[blockIdx.x];
    const int L = P.faceL[f], R = P.faceR[f];
    const int Nv = P.Nv, Nvp = P.Nvp;
    double An[3] = {0, 0, 0}, rl[3] = {0, 0, 0}, rr[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) {
        An[d] = P.An[(size_t)f * D + d];
        rl[d] = P.rL[(size_t)f * D + d];
        if (R >= 0) rr[d] = P.rR[(size_t)f * D + d];
    }
    T* fx = P.FX + (size_t)f * NA * Nvp;
    const size_t cs = (size_t)NA * Nvp;
    int btype = 0;
    double rb = 0.0, Ub[3] = {0, 0, 0}, RTb = 0.0;
    if (R < 0) {
        const double* B = P.bc + (size_t)(-1 - R) * 6;
        btype = (int)B[0];
        rb = B[1];
        for (int d = 0; d < 3; ++d) Ub[d] = B[2 + d];
        RTb = P.g.R * B[5];
    }
    // pass A: foot values phi_C + (L grad phi)_C . (r_C - xi h), C upwind by xi . n
    double acc[NW];
#pragma unroll
    for (int m = 0; m < NW; ++m) acc[m] = 0.0;
    for (int k = threadIdx.x; k < Nv; k += RK_NT) {
        double x[3] = {0, 0, 0}, x2 = 0.0;
        for (int d = 0; d < D; ++d) {
            x[d] = P.xi[(size_t)k * D + d];
            x2 += x[d] * x[d];
        }
        // xi . A n without contraction: the upwind decision is taken exactly as in a plain FP64 code
        const double sn = dot_rn<D>(x, An);
        const int C = sn >= 0.0 ? L : R;
        const double* r = sn >= 0.0 ? rl : rr;
        T ph[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) ph[a] = T(0);
        if (C >= 0) {
            T off[D];
#pragma unroll
            for (int d = 0; d < D; ++d) off[d] = (T)(r[d] - x[d] * P.h);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                T v = P.f[(size_t)C * cs + (size_t)a * Nvp + k];
                if (P.G)
#pragma unroll
                    for (int d = 0; d < D; ++d) v += P.G[(((size_t)C * NA + a) * D + d) * Nvp + k] * off[d];
                ph[a] = v;
            }
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) fx[(size_t)a * Nvp + k] = ph[a];
        const double wk = P.w[k];
        if (R >= 0) {
            const double G = (double)ph[0], H = D == 2 ? (double)ph[1] : 0.0, Rr = (double)ph[NA - 1];
            acc[0] += wk * G;
            for (int d = 0; d < D; ++d) acc[1 + d] += wk * x[d] * G;
            acc[D + 1] += wk * (0.5 * (x2 * G + H) + Rr);
            acc[D + 2] += wk * Rr;
        } else if (btype == AVS_BC_WALL) {
            if (sn >= 0.0) {
                acc[0] += wk * sn * (double)ph[0];
            } else {
                double c2 = 0.0;
                for (int d = 0; d < D; ++d) c2 += (x[d] - Ub[d]) * (x[d] - Ub[d]);
                acc[1] += wk * (-sn) * (1.0 / pow(2.0 * AVS_PI * RTb, 0.5 * D) * exp(-c2 / (2.0 * RTb)));
            }
        }
    }
    block_sum<NW, RK_NT>(acc, sred, sout);
    if (R >= 0) {
        double W[NW];
#pragma unroll
        for (int m = 0; m < NW; ++m) W[m] = sout[m];
        double U[D], a2[2 * D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            U[d] = W[1 + d] / W[0];
            a2[d] = a2[D + d] = 0.0;
        }
        for (int k = threadIdx.x; k < Nv; k += RK_NT) {
            const double wk = P.w[k];
            double c[D], c2 = 0.0;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                c[d] = P.xi[(size_t)k * D + d] - U[d];
                c2 += c[d] * c[d];
            }
            const double G = (double)fx[k], H = D == 2 ? (double)fx[Nvp + k] : 0.0;
            const double Rr = (double)fx[(size_t)(NA - 1) * Nvp + k];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                a2[d] += 0.5 * wk * c[d] * (c2 * G + H);
                a2[D + d] += wk * c[d] * Rr;
            }
        }
        block_sum<2 * D, RK_NT>(a2, sred, sout);
        if (threadIdx.x == 0) {
            double rho, Uu[3], RTt, RTr, RT;
            rk_prim<D>(W, rho, Uu, RTt, RTr, RT);
            if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
            const double tau = rk_tau(P.g, rho, RTt);
            // rotational energy relaxed over h toward rho R T, T fixed by the total energy
            const double az = P.h / (P.g.Z * tau);
            RTr = (W[D + 2] + az * rho * RT) / (1.0 + az) / rho;
            RTt = (5.0 * RT - 2.0 * RTr) / 3.0;
            const double lt = 2.0 / 3.0 + (1.0 - P.g.om0) / (3.0 * P.g.Z);
            const double lr = 1.0 - (1.0 - P.g.dl) * ((1.0 - 1.0 / P.g.Z) * RTr / RTt + P.g.om1 / P.g.Z);
            double qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                qt[d] = tau * sout[d] / (tau + P.h * lt);
                qr[d] = tau * sout[D + d] / (tau + P.h * lr);
            }
            eq = rk_make<D, T>(P.g, rho, Uu, RTt, RTr, qt, qr);
            blend[0] = tau / (tau + P.h);
            blend[1] = P.h / (tau + P.h);
        }
    } else if (threadIdx.x == 0) {
        // incoming half: rho_b g^eq(U_b, T_b) with H = (3 - D) R T_b G, R = R T_b G
        const double rho_b = btype == AVS_BC_WALL ? (sout[1] > 0.0 ? sout[0] / sout[1] : 0.0) : rb;
        const double z[3] = {0, 0, 0};
        RkGas g0 = P.g;
        g0.iz = 0.0;
        eq = rk_make<D, T>(g0, rho_b, Ub, RTb, RTb, z, z);
        blend[0] = 1.0;
        blend[1] = 0.0;
    }
    __syncthreads();
    // pass B: phi_ij, per-node flux (xi . A n) phi and its moments
    const T wa = blend[0], wb = blend[1];
    double af[NW];
#pragma unroll
    for (int m = 0; m < NW; ++m) af[m] = 0.0;
    for (int k = threadIdx.x; k < Nv; k += RK_NT) {
        double x[3] = {0, 0, 0}, x2 = 0.0;
        T xt[D];
        for (int d = 0; d < D; ++d) {
            x[d] = P.xi[(size_t)k * D + d];
            x2 += x[d] * x[d];
            xt[d] = (T)x[d];
        }
        const double sn = dot_rn<D>(x, An);
        T ph[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) ph[a] = fx[(size_t)a * Nvp + k];
        if (R >= 0 || sn < 0.0) {
            T gv[NA];
            rk_eval<D, T>(eq, xt, gv);
#pragma unroll
            for (int a = 0; a < NA; ++a) ph[a] = R >= 0 ? wa * ph[a] + wb * gv[a] : gv[a];
        }
        const T st = (T)sn;
        double Fd[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const T F = st * ph[a];
            fx[(size_t)a * Nvp + k] = F;
            Fd[a] = (double)F;
        }
        const double wk = P.w[k];
        af[0] += wk * Fd[0];
        for (int d = 0; d < D; ++d) af[1 + d] += wk * x[d] * Fd[0];
        af[D + 1] += wk * (0.5 * (x2 * Fd[0] + (D == 2 ? Fd[1] : 0.0)) + Fd[NA - 1]);
        af[D + 2] += wk * Fd[NA - 1];
    }
    block_sum<NW, RK_NT>(af, sred, sout);
    if (threadIdx.x < NW) P.AF[(size_t)f * NW + threadIdx.x] = sout[threadIdx.x];
}

// One cell: W~ = W - dt/|V| sum A F with the rotational source of Eq. (S_rot)
// taken implicitly, tau from T_t of the flux-updated state (reading R28);
// lagged heat fluxes of f^n (R3); the collision update of every array.
template <int D, typename T>
__global__ void __launch_bounds__(RK_NT) rk_cell(RkP<T> P)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3;
    __shared__ double sred[(RK_NT / 32) * 6], sout[6];
    __shared__ RkEq<T> eq;
    __shared__ double tau_s;
    __shared__ int fs[AVS_MAXS];
    __shared__ T sg[AVS_MAXS];
    const int i = blockIdx.x;
    const int ns = P.nslot[i];
    const int Nv = P.Nv, Nvp = P.Nvp;
    if (threadIdx.x < ns) {
        const int sl = P.slot[i * AVS_MAXS + threadIdx.x];
        fs[threadIdx.x] = sl >> 1;
        sg[threadIdx.x] = (sl & 1) ? T(-1) : T(1);
    }
    const size_t cs = (size_t)NA * Nvp;
    const T* fi = P.f + (size_t)i * cs;
    double Wn[NW], qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
    rk_cell_mom<D, T>(fi, Nv, Nvp, P.xi, P.w, Wn, qt, qr, sred, sout);
    if (threadIdx.x == 0) {
        const double V = P.vol[i];
        double Wt[NW];
        for (int c = 0; c < NW; ++c) {
            double s = 0.0;
            for (int q = 0; q < ns; ++q) {
                const double a = P.AF[(size_t)fs[q] * NW + c];
                s += sg[q] > T(0) ? a : -a;
            }
            Wt[c] = P.Win[(size_t)i * NW + c] - P.dt / V * s;
        }
        double rho, U[3], RTt, RTr, RT;
        rk_prim<D>(Wt, rho, U, RTt, RTr, RT);
        if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
        const double tau = rk_tau(P.g, rho, RTt);
        const double az = P.dt / (P.g.Z * tau);
        Wt[D + 2] = (Wt[D + 2] + az * rho * RT) / (1.0 + az);
        rk_prim<D>(Wt, rho, U, RTt, RTr, RT);
        eq = rk_make<D, T>(P.g, rho, U, RTt, RTr, qt, qr);
        tau_s = tau;
        for (int c = 0; c < NW; ++c) P.Wout[(size_t)i * NW + c] = Wt[c];
    }
    __syncthreads();
    const T dt = (T)P.dt, tau = (T)tau_s, V = (T)P.vol[i];
    const T den = T(1) / dt + T(1) / tau;
    T* fo = P.fout + (size_t)i * cs;
    for (int k = threadIdx.x; k < Nvp; k += RK_NT) {
        if (k >= Nv) {
#pragma unroll
            for (int a = 0; a < NA; ++a) fo[(size_t)a * Nvp + k] = T(0);
            continue;
        }
        T xt[D];
#pragma unroll
        for (int d = 0; d < D; ++d) xt[d] = (T)P.xi[(size_t)k * D + d];
        T gv[NA];
        rk_eval<D, T>(eq, xt, gv);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            T N = T(0);
            for (int q = 0; q < ns; ++q) N += sg[q] * P.FX[((size_t)fs[q] * NA + a) * Nvp + k];
            fo[(size_t)a * Nvp + k] = (fi[(size_t)a * Nvp + k] / dt + gv[a] / tau - N / V) / den;
        }
    }
}

// ---------------------------------------------------------------- mixed form
// The FP32 form sums over the nodes in FP32 per thread (FP64 across warps),
// as raw moments about a reference velocity V near the local mean velocity
// (the upwind-side cell's carried U), so that no per-node FP64 arithmetic is
// left: on GB300 an FP64 operation costs about as much as 70 FP32 ones.

template <int D>
struct RkNR {
    static constexpr int v = D == 2 ? 14 : 17;
};

// Raw moments of one node about V (c = xi - V): w G; w c_d G; w c_d c_e G
// (d <= e); w c_d c^2 G; in 2D w H and w c_d H; w R and w c_d R.
template <int D>
__device__ __forceinline__ void rk_raw_acc(float* m, const float* c, float wG, float wH, float wR)
{
    int o = 0;
    float c2 = 0.0f;
#pragma unroll
    for (int d = 0; d < D; ++d) c2 += c[d] * c[d];
    m[o++] += wG;
#pragma unroll
    for (int d = 0; d < D; ++d) m[o++] += c[d] * wG;
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
        for (int e = d; e < D; ++e) m[o++] += c[d] * c[e] * wG;
#pragma unroll
    for (int d = 0; d < D; ++d) m[o++] += c[d] * c2 * wG;
    if (D == 2) {
        m[o++] += wH;
#pragma unroll
        for (int d = 0; d < D; ++d) m[o++] += c[d] * wH;
    }
    m[o++] += wR;
#pragma unroll
    for (int d = 0; d < D; ++d) m[o++] += c[d] * wR;
}

// W = (rho, rho U, rho E, rho E_rot) and, when qt is given, the heat fluxes
// about U (Eq. 8) from the raw moments about V: with delta = U - V,
// c' = c - delta, sum w c'_i c'^2 G = m3_i - 2 delta_j m2_ij + delta^2 m1_i
// - delta_i tr m2 + 2 delta_i (delta . m1) - delta_i delta^2 m0.
template <int D>
__device__ void rk_from_raw(const double* m, const double* V, double* W, double* qt, double* qr)
{
    int o = 0;
    const double m0 = m[o++];
    double m1[3] = {0, 0, 0}, m2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, m3[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) m1[d] = m[o++];
    for (int d = 0; d < D; ++d)
        for (int e = d; e < D; ++e) m2[d][e] = m2[e][d] = m[o++];
    for (int d = 0; d < D; ++d) m3[d] = m[o++];
    double h0 = 0.0, h1[3] = {0, 0, 0};
    if (D == 2) {
        h0 = m[o++];
        for (int d = 0; d < D; ++d) h1[d] = m[o++];
    }
    const double r0 = m[o++];
    double r1[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) r1[d] = m[o++];
    const double rho = m0;
    double dl[3] = {0, 0, 0}, d2 = 0.0, tr = 0.0, VV = 0.0, Vm = 0.0, dm = 0.0;
    for (int d = 0; d < D; ++d) {
        dl[d] = m1[d] / rho;
        d2 += dl[d] * dl[d];
        tr += m2[d][d];
        VV += V[d] * V[d];
        Vm += V[d] * m1[d];
        dm += dl[d] * m1[d];
    }
    W[0] = rho;
    for (int d = 0; d < D; ++d) W[1 + d] = rho * V[d] + m1[d];
    W[D + 1] = 0.5 * (VV * m0 + 2.0 * Vm + tr + h0) + r0;
    W[D + 2] = r0;
    if (!qt) return;
    for (int i = 0; i < D; ++i) {
        double s = m3[i] + d2 * m1[i] - dl[i] * tr + 2.0 * dl[i] * dm - dl[i] * d2 * m0;
        for (int j = 0; j < D; ++j) s -= 2.0 * dl[j] * m2[i][j];
        qt[i] = 0.5 * (s + (h1[i] - dl[i] * h0));
        qr[i] = r1[i] - dl[i] * r0;
    }
}

// FP32 state of the raw moments about V (the mixed form's per-face and
// per-cell parameters; FP64 is 70x scarcer than FP32 on GB300): rho, U, the
// translational internal energy (with H) e_t = (sum w (c'^2 G + H))/2 about
// U, the rotational energy r0 and the heat fluxes, all from the centred
// sums, so that no bulk kinetic energy cancels.
template <int D>
__device__ void rk_state_raw32(const double* md, const double* V, float& rho, float* U, float& et, float& r0,
                               float* qt, float* qr)
{
    constexpr int NR = RkNR<D>::v;
    float m[NR];
    for (int q = 0; q < NR; ++q) m[q] = (float)md[q];
    int o = 0;
    const float m0 = m[o++];
    float m1[3] = {0, 0, 0}, m2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, m3[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) m1[d] = m[o++];
    for (int d = 0; d < D; ++d)
        for (int e = d; e < D; ++e) m2[d][e] = m2[e][d] = m[o++];
    for (int d = 0; d < D; ++d) m3[d] = m[o++];
    float h0 = 0.0f, h1[3] = {0, 0, 0};
    if (D == 2) {
        h0 = m[o++];
        for (int d = 0; d < D; ++d) h1[d] = m[o++];
    }
    r0 = m[o++];
    float r1[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) r1[d] = m[o++];
    rho = m0;
    const float ir = 1.0f / m0;
    float dl[3] = {0, 0, 0}, d2 = 0.0f, tr = 0.0f, dm = 0.0f;
    for (int d = 0; d < D; ++d) {
        dl[d] = m1[d] * ir;
        U[d] = (float)V[d] + dl[d];
        d2 += dl[d] * dl[d];
        tr += m2[d][d];
        dm += dl[d] * m1[d];
    }
    et = 0.5f * (tr + h0 - m0 * d2);
    for (int i = 0; i < D; ++i) {
        float s = m3[i] + d2 * m1[i] - dl[i] * tr + 2.0f * dl[i] * dm - dl[i] * d2 * m0;
        for (int j = 0; j < D; ++j) s -= 2.0f * dl[j] * m2[i][j];
        qt[i] = 0.5f * (s + (h1[i] - dl[i] * h0));
        qr[i] = r1[i] - dl[i] * r0;
    }
}

// RkEq<float> of a state given in FP32, without FP64 arithmetic.
template <int D>
__device__ RkEq<float> rk_make32(const RkGas& g, float rho, const float* U, float RTt, float RTr, const float* qt,
                                 const float* qr)
{
    RkEq<float> e;
    const float RT = (3.0f * RTt + 2.0f * RTr) * 0.2f;
    const float pt = rho * RTt, p = rho * RT;
    const float om0 = (float)g.om0, om1 = (float)g.om1, dl = (float)g.dl;
    for (int d = 0; d < 3; ++d) {
        const bool on = d < D;
        e.U[d] = on ? U[d] : 0.0f;
        e.at[d] = on ? qt[d] / (15.0f * pt * RTt) : 0.0f;
        e.ar[d] = on ? om0 * qt[d] / (15.0f * p * RT) : 0.0f;
        e.bt[d] = on ? (1.0f - dl) * qr[d] / (pt * RTt) : 0.0f;
        e.br[d] = on ? om1 * (1.0f - dl) * qr[d] / (p * RT) : 0.0f;
    }
    const float xt = 2.0f * (float)AVS_PI * RTt, xr = 2.0f * (float)AVS_PI * RT;
    e.pt = D == 2 ? rho / xt : rho / (xt * sqrtf(xt));
    e.pr = D == 2 ? rho / xr : rho / (xr * sqrtf(xr));
    e.RTt = RTt;
    e.RTr = RTr;
    e.RT = RT;
    e.iRTt = 1.0f / RTt;
    e.iRT = 1.0f / RT;
    e.iz = (float)g.iz;
    return e;
}

// tau = mu(T_t) / p_t in FP32
__device__ __forceinline__ float rk_tau32(const RkGas& g, float rho, float RTt)
{
    const float T = RTt / (float)g.R;
    return (float)g.mu_ref * powa(T / (float)g.T_ref, (float)g.omega) / (rho * RTt);
}

// The FP64 upwind decision (the oracle's) for the nodes inside the FP32
// rounding bound.  Not inlined: inlined, the compiler predicates it into every
// node's instruction stream, and an FP64 instruction issued with its predicate
// off still occupies the scarce FP64 pipe (out of line, the face kernel's FP64
// pipe went from 52 % to 4 % busy and the kernel ran 12 % faster).
template <int D>
__device__ __noinline__ bool rk_upwind_exact(const double* __restrict__ xi, int k, const double* An)
{
    double xd[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) xd[d] = xi[(size_t)k * D + d];
    return dot_rn<D>(xd, An) >= 0.0;
}

// Upwind side of a node: xi . A n >= 0 decided in FP32 when the FP32 sum is
// farther from zero than its rounding bound, else in FP64 without
// contraction, so the decision always equals the FP64 one.
template <int D>
__device__ __forceinline__ bool rk_upwind_L(const float* x, const float* Af, const double* __restrict__ xi, int k,
                                            const double* An, float& s)
{
    float a = 0.0f;
    s = 0.0f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float p = __fmul_rn(x[d], Af[d]);
        s = __fadd_rn(s, p);
        a += fabsf(p);
    }
    if (fabsf(s) > a * 0x1p-20f) return s >= 0.0f;
    return rk_upwind_exact<D>(xi, k, An);
}

// rk_face for the FP32 form (same steps; sums as above).
template <int D>
__global__ void __launch_bounds__(RK_NT, D == 2 ? 8 : 7) rk_face32(RkP<float> P, const float* __restrict__ xif,
                                                   const float* __restrict__ wf, const float* __restrict__ Anf,
                                                   const float* __restrict__ rLf, const float* __restrict__ rRf)
{
    using T = float;
    constexpr int NA = RkNA<D>::v, NW = D + 3, NR = RkNR<D>::v;
    __shared__ double sw[(RK_NT / 32) * RkNR<3>::v], sout[RkNR<3>::v];
    __shared__ RkEq<T> eq;
    __shared__ float blend[2];
    // per-face constants, converted from FP64 once by thread 0 (an FP64
    // conversion or division in every thread costs as much as the node work)
    __shared__ float cAf[3], crl[3], crr[3], cV[3], cUb[3], cpw, ci2b, ch;
    __shared__ double An[3], Vd[3], cRTb, crb;
    __shared__ int cbt;
    const int f = P.order[blockIdx.x];
    const int L = P.faceL[f], R = P.faceR[f];
    const int Nv = P.Nv, Nvp = P.Nvp;
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) {
            An[d] = d < D ? P.An[(size_t)f * D + d] : 0.0;
            cAf[d] = d < D ? Anf[(size_t)f * D + d] : 0.0f;
            crl[d] = d < D ? rLf[(size_t)f * D + d] : 0.0f;
            crr[d] = d < D && R >= 0 ? rRf[(size_t)f * D + d] : 0.0f;
        }
        int btype = 0;
        double rb = 0.0, Ub[3] = {0, 0, 0}, RTb = 1.0;
        if (R < 0) {
            const double* B = P.bc + (size_t)(-1 - R) * 6;
            btype = (int)B[0];
            rb = B[1];
            for (int d = 0; d < 3; ++d) Ub[d] = B[2 + d];
            RTb = P.g.R * B[5];
        }
        cbt = btype;
        crb = rb;
        cRTb = RTb;
        // reference velocity of the sums: the left cell's mean velocity in
        // FP32 (any V gives the same moments; Vd is its exact FP64 value)
        const double* WL = P.Win + (size_t)L * NW;
        const float irL = 1.0f / (float)WL[0];
        for (int d = 0; d < 3; ++d) {
            cV[d] = d < D ? (float)WL[1 + d] * irL : 0.0f;
            Vd[d] = (double)cV[d];
            cUb[d] = (float)Ub[d];
        }
        // wall Maxwellian prefactor (2 pi RT_w)^(-D/2) and 1/(2 RT_w) in FP32
        const float xb = 2.0f * (float)AVS_PI * (float)RTb;
        cpw = D == 2 ? 1.0f / xb : 1.0f / (xb * sqrtf(xb));
        ci2b = 0.5f / (float)RTb;
        ch = (float)P.h;
    }
    __syncthreads();
    T Af[D], rl[D], rr[D], V[D], Ubf[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        Af[d] = cAf[d];
        rl[d] = crl[d];
        rr[d] = crr[d];
        V[d] = cV[d];
        Ubf[d] = cUb[d];
    }
    const int btype = cbt;
    const T pw = cpw, i2b = ci2b;
    T* fx = P.FX + (size_t)f * NA * Nvp;
    const size_t cs = (size_t)NA * Nvp;
    const T h = ch;
    T racc[NR], wacc[2] = {T(0), T(0)};
#pragma unroll
    for (int m = 0; m < NR; ++m) racc[m] = T(0);
    // pass A: foot values and their raw moments (or the wall balance); the
    // interior and boundary loops are separate so that neither carries the
    // other's instructions predicated off
    const int Rc = R >= 0 ? R : L;
    const float* fLp = P.f + (size_t)L * cs;
    const float* fRp = P.f + (size_t)Rc * cs;
    const float* gLp = P.G ? P.G + (size_t)L * NA * D * Nvp : nullptr;
    const float* gRp = P.G ? P.G + (size_t)Rc * NA * D * Nvp : nullptr;
    if (R >= 0) {
        for (int k = threadIdx.x; k < Nv; k += RK_NT) {
            T x[D];
#pragma unroll
            for (int d = 0; d < D; ++d) x[d] = xif[(size_t)k * D + d];
            T s;
            const bool up = rk_upwind_L<D>(x, Af, P.xi, k, An, s);
            const float* fb = (up ? fLp : fRp) + k;
            T ph[NA];
            if (gLp) {
                const float* gb = (up ? gLp : gRp) + k;
                T off[D];
#pragma unroll
                for (int d = 0; d < D; ++d) off[d] = (up ? rl[d] : rr[d]) - x[d] * h;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    T v = fb[a * Nvp];
#pragma unroll
                    for (int d = 0; d < D; ++d) v += gb[(a * D + d) * Nvp] * off[d];
                    ph[a] = v;
                }
            } else {
#pragma unroll
                for (int a = 0; a < NA; ++a) ph[a] = fb[a * Nvp];
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) fx[(size_t)a * Nvp + k] = ph[a];
            const T wk = wf[k];
            T c[D];
#pragma unroll
            for (int d = 0; d < D; ++d) c[d] = x[d] - V[d];
            rk_raw_acc<D>(racc, c, wk * ph[0], D == 2 ? wk * ph[1] : T(0), wk * ph[NA - 1]);
        }
    } else {
        for (int k = threadIdx.x; k < Nv; k += RK_NT) {
            T x[D];
#pragma unroll
            for (int d = 0; d < D; ++d) x[d] = xif[(size_t)k * D + d];
            T s;
            const bool up = rk_upwind_L<D>(x, Af, P.xi, k, An, s);
            T ph[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) ph[a] = T(0);
            if (up) {
                T off[D];
#pragma unroll
                for (int d = 0; d < D; ++d) off[d] = rl[d] - x[d] * h;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    T v = fLp[a * Nvp + k];
                    if (gLp)
#pragma unroll
                        for (int d = 0; d < D; ++d) v += gLp[(a * D + d) * Nvp + k] * off[d];
                    ph[a] = v;
                }
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) fx[(size_t)a * Nvp + k] = ph[a];
            if (btype == AVS_BC_WALL) {
                const T wk = wf[k];
                if (up) {
                    wacc[0] += wk * s * ph[0];
                } else {
                    T c2 = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) c2 += (x[d] - Ubf[d]) * (x[d] - Ubf[d]);
                    wacc[1] += wk * (-s) * (pw * ex(-c2 * i2b));
                }
            }
        }
    }
    if (R >= 0) {
        block_sum_t<NR, RK_NT>(racc, sw, sout);
        if (threadIdx.x == 0) {
            // the interface state in FP32 (as the monatomic mixed form): no FP64 pow or division here
            float rho, Uu[3] = {0, 0, 0}, et, r0, qb[3] = {0, 0, 0}, qrb[3] = {0, 0, 0};
            rk_state_raw32<D>(sout, Vd, rho, Uu, et, r0, qb, qrb);
            float RTt = et / (1.5f * rho), RT = (et + r0) / (2.5f * rho);
            if (!(rho > 0.0f) || !(RTt > 0.0f) || !(RT > 0.0f)) atomicOr(P.err, 1);
            const float tau = rk_tau32(P.g, rho, RTt), hf = (float)P.h, Z = (float)P.g.Z;
            const float az = hf / (Z * tau);
            const float RTr = (r0 + az * rho * RT) / (1.0f + az) / rho;
            RTt = (5.0f * RT - 2.0f * RTr) * (1.0f / 3.0f);
            const float lt = 2.0f / 3.0f + (1.0f - (float)P.g.om0) / (3.0f * Z);
            const float lr = 1.0f - (1.0f - (float)P.g.dl) * ((1.0f - 1.0f / Z) * RTr / RTt + (float)P.g.om1 / Z);
            float qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) {
                qt[d] = tau * qb[d] / (tau + hf * lt);
                qr[d] = tau * qrb[d] / (tau + hf * lr);
            }
            eq = rk_make32<D>(P.g, rho, Uu, RTt, RTr, qt, qr);
            blend[0] = tau / (tau + hf);
            blend[1] = hf / (tau + hf);
        }
    } else {
        block_sum_t<2, RK_NT>(wacc, sw, sout);
        if (threadIdx.x == 0) {
            const double rho_b = btype == AVS_BC_WALL ? (sout[1] > 0.0 ? sout[0] / sout[1] : 0.0) : crb;
            const double z[3] = {0, 0, 0};
            const double* B = P.bc + (size_t)(-1 - R) * 6;
            const double Ub[3] = {B[2], B[3], B[4]};
            RkGas g0 = P.g;
            g0.iz = 0.0;
            eq = rk_make<D, T>(g0, rho_b, Ub, cRTb, cRTb, z, z);
            blend[0] = 1.0;
            blend[1] = 0.0;
        }
    }
    __syncthreads();
    // pass B: phi_ij, per-node flux (xi . A n) phi and its moments
    const T wa = (T)blend[0], wb = (T)blend[1];
    T af[NW];
#pragma unroll
    for (int m = 0; m < NW; ++m) af[m] = T(0);
    // interior: phi = wa phi_bar + wb g at every node; boundary: the
    // incoming nodes take g (wall or far-field Maxwellian)
    const bool inter = R >= 0;
    for (int k = threadIdx.x; k < Nv; k += RK_NT) {
        T x[D], x2 = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            x[d] = xif[(size_t)k * D + d];
            x2 += x[d] * x[d];
        }
        T s;
        const bool up = rk_upwind_L<D>(x, Af, P.xi, k, An, s);
        T ph[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) ph[a] = fx[(size_t)a * Nvp + k];
        if (inter) {
            T gv[NA];
            rk_eval<D, T>(eq, x, gv);
#pragma unroll
            for (int a = 0; a < NA; ++a) ph[a] = wa * ph[a] + wb * gv[a];
        } else if (!up) {
            T gv[NA];
            rk_eval<D, T>(eq, x, gv);
#pragma unroll
            for (int a = 0; a < NA; ++a) ph[a] = gv[a];
        }
        T F[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            F[a] = s * ph[a];
            fx[(size_t)a * Nvp + k] = F[a];
        }
        const T wk = wf[k];
        af[0] += wk * F[0];
#pragma unroll
        for (int d = 0; d < D; ++d) af[1 + d] += wk * x[d] * F[0];
        af[D + 1] += wk * (T(0.5) * (x2 * F[0] + (D == 2 ? F[1] : T(0))) + F[NA - 1]);
        af[D + 2] += wk * F[NA - 1];
    }
    block_sum_t<NW, RK_NT>(af, sw, sout);
    if (threadIdx.x < NW) P.AF[(size_t)f * NW + threadIdx.x] = sout[threadIdx.x];
}

// ---------------------------------------------------------------- mixed-form cell stage
// As the monatomic mixed form: the raw moments of f^{n+1} that the next step
// needs for its lagged heat fluxes are summed while f^{n+1} is written and
// carried per cell ([cell][NR] FP64, about V(W^{n+1})); all per-cell FP64
// work (the balance of W, the rotational relaxation) runs one thread per
// cell in rk_cell_state32; the cell kernel streams f, the face fluxes and
// f^{n+1} RK_VC nodes per thread in vector loads.

// Per-cell parameters of the Rykov collision update (mixed form).
struct RkCellPar {
    RkEq<float> eq;          // Rykov equilibrium of (W~ with relaxed E_rot, q~)
    float upd[4];            // 1/dt, 1/tau~, 1/|V|, 1/(1/dt + 1/tau~)
    float Vn[3];             // reference velocity of the next raw moments: V(W^{n+1})
};
static_assert(sizeof(RkCellPar) <= AVS_CELLPAR_BYTES, "RkCellPar buffer size");
static_assert(RkNR<3>::v <= AVS_CMOM_MAX, "carried moments buffer size");

constexpr int RK_VC = 2;     // nodes per thread per iteration of the cell kernels (2 or 4)

// Reference velocity of the raw sums of a cell from a carried W (FP32; the
// same expression wherever carried moments are taken or used).
template <int D>
__device__ __forceinline__ void rk_vref(const double* W, float* V)
{
    const float ir = 1.0f / (float)W[0];
#pragma unroll
    for (int d = 0; d < 3; ++d) V[d] = d < D ? (float)W[1 + d] * ir : 0.0f;
}

// V = RK_VC consecutive nodes of an FP32 row in one vector load (L2 only).
__device__ __forceinline__ void rk_ldv(const float* p, float* o)
{
    if constexpr (RK_VC == 4) {
        const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    } else {
        const float2 t = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = t.x;
        o[1] = t.y;
    }
}

__device__ __forceinline__ void rk_stv(float* p, const float* o)
{
    if constexpr (RK_VC == 4)
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    else
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
}

// xi (D per node) and w of the RK_VC nodes from k0 (rows padded to 32 nodes;
// k0 is a multiple of RK_VC, so the vectors are aligned).
template <int D>
__device__ __forceinline__ void rk_ld_nodes(const float* __restrict__ xif, const float* __restrict__ wf, int k0,
                                            float (*x)[D], float* w)
{
    constexpr int V = RK_VC;
    float t[V * D];
#pragma unroll
    for (int j = 0; j < V * D / 2; ++j) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(xif + (size_t)k0 * D) + j);
        t[2 * j] = q.x;
        t[2 * j + 1] = q.y;
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
        for (int d = 0; d < D; ++d) x[v][d] = t[v * D + d];
#pragma unroll
    for (int j = 0; j < V / 2; ++j) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(wf + k0) + j);
        w[2 * j] = q.x;
        w[2 * j + 1] = q.y;
    }
}

// Raw moments of the own f^n of every cell about V(W^n), when the previous
// step did not leave them (after init, set_f, an adaptation or an implicit
// step).  Same nodes per thread and order as rk_cell32, so the sums are the
// carried ones bit for bit.
template <int D>
__global__ void __launch_bounds__(RK_NT) rk_raw_moments32(RkP<float> P, const float* __restrict__ xif,
                                                          const float* __restrict__ wf, double* mom)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3, NR = RkNR<D>::v;
    __shared__ double sw[(RK_NT / 32) * NR], red[NR];
    const int i = blockIdx.x;
    const int Nvp = P.Nvp;
    float V[3];
    rk_vref<D>(P.Win + (size_t)i * NW, V);
    const float* fi = P.f + (size_t)i * NA * Nvp;
    float acc[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) acc[m] = 0.0f;
    for (int k0 = threadIdx.x * RK_VC; k0 < P.Nv; k0 += RK_NT * RK_VC) {
        float x[RK_VC][D], wv[RK_VC], fv[NA][RK_VC];
        rk_ld_nodes<D>(xif, wf, k0, x, wv);
#pragma unroll
        for (int a = 0; a < NA; ++a) rk_ldv(fi + (size_t)a * Nvp + k0, fv[a]);
#pragma unroll
        for (int v = 0; v < RK_VC; ++v) {
            float c[D];
#pragma unroll
            for (int d = 0; d < D; ++d) c[d] = x[v][d] - V[d];
            rk_raw_acc<D>(acc, c, wv[v] * fv[0][v], D == 2 ? wv[v] * fv[1][v] : 0.0f, wv[v] * fv[NA - 1][v]);
        }
    }
    block_sum_t<NR, RK_NT>(acc, sw, red);
    if (threadIdx.x < NR) mom[(size_t)i * NR + threadIdx.x] = red[threadIdx.x];
}

// One thread per cell: lagged q_t, q_r of f^n from its carried moments,
// W~ = W - dt/|V| sum_j sgn_j A F_j (FP64), the implicit rotational relaxation
// of E_rot over dt with tau~ (reading R28), and the collision parameters.
template <int D>
__global__ void rk_cell_state32(RkP<float> P, const double* __restrict__ mom, RkCellPar* par)
{
    constexpr int NW = D + 3, NR = RkNR<D>::v;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.Nc) return;
    const double* Wi = P.Win + (size_t)i * NW;
    float V[3];
    rk_vref<D>(Wi, V);
    const double Vd[3] = {V[0], V[1], V[2]};
    float rn, Un[3], etn, r0n, qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
    rk_state_raw32<D>(mom + (size_t)i * NR, Vd, rn, Un, etn, r0n, qt, qr);
    const int ns = P.nslot[i];
    const double dtV = P.dt / P.vol[i];
    double Wt[NW];
    for (int c = 0; c < NW; ++c) {
        double sum = 0.0;
        for (int q = 0; q < ns; ++q) {
            const int sl = P.slot[i * AVS_MAXS + q];
            const double a = P.AF[(size_t)(sl >> 1) * NW + c];
            sum += (sl & 1) ? -a : a;
        }
        Wt[c] = Wi[c] - dtV * sum;
    }
    const double rho = Wt[0], ir = 1.0 / rho;
    double m2 = 0.0;
    float U[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) {
        m2 += Wt[1 + d] * Wt[1 + d];
        U[d] = (float)(Wt[1 + d] * ir);
    }
    const double ein = Wt[D + 1] - 0.5 * m2 * ir;   // rho e, translational + rotational
    const double RT = ein * ir * 0.4, RTt = (ein - Wt[D + 2]) * ir * (1.0 / 1.5);
    if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
    const float tau = rk_tau32(P.g, (float)rho, (float)RTt);
    const double az = P.dt / (P.g.Z * (double)tau);
    Wt[D + 2] = (Wt[D + 2] + az * rho * RT) / (1.0 + az);
    const double RTr = Wt[D + 2] * ir;
    for (int c = 0; c < NW; ++c) P.Wout[(size_t)i * NW + c] = Wt[c];
    RkCellPar cp;
    cp.eq = rk_make32<D>(P.g, (float)rho, U, (float)((5.0 * RT - 2.0 * RTr) * (1.0 / 3.0)), (float)RTr, qt, qr);
    const float dtf = (float)P.dt, idt = 1.0f / dtf, itau = 1.0f / tau;
    cp.upd[0] = idt;
    cp.upd[1] = itau;
    cp.upd[2] = 1.0f / (float)P.vol[i];
    cp.upd[3] = dtf * tau / (dtf + tau);
    rk_vref<D>(Wt, cp.Vn);
    par[i] = cp;
}

// One block per cell: net flux N = sum_j sgn_j F_j per node, the collision
// update (Eq. SGS_phi's diagonal, R1) with the Rykov equilibrium, pad nodes
// written as zero, and the raw moments of f^{n+1} about V(W^{n+1}) for the
// next step.
template <int D>
__global__ void __launch_bounds__(RK_NT, 7) rk_cell32(RkP<float> P, const float* __restrict__ xif,
                                                   const float* __restrict__ wf, double* mom,
                                                   const RkCellPar* __restrict__ par)
{
    constexpr int NA = RkNA<D>::v, NR = RkNR<D>::v, V = RK_VC;
    __shared__ double sw[(RK_NT / 32) * NR], red[NR];
    __shared__ RkCellPar cp;
    __shared__ int fs[AVS_MAXS];
    __shared__ float sg[AVS_MAXS];
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int ns = P.nslot[i];
    const int Nv = P.Nv, Nvp = P.Nvp;
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        fs[tid] = sl >> 1;
        sg[tid] = (sl & 1) ? -1.0f : 1.0f;
    }
    if (tid == 32) cp = par[i];
    __syncthreads();
    const size_t cs = (size_t)NA * Nvp;
    const float* fi = P.f + (size_t)i * cs;
    float* fo = P.fout + (size_t)i * cs;
    const float u0 = cp.upd[0], u1 = cp.upd[1], u2 = cp.upd[2], u3 = cp.upd[3];
    float Vn[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vn[d] = cp.Vn[d];
    float acc[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) acc[m] = 0.0f;
    for (int k0 = tid * V; k0 < Nv; k0 += RK_NT * V) {
        float x[V][D], wv[V], fv[NA][V], Nn[NA][V];
        rk_ld_nodes<D>(xif, wf, k0, x, wv);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            rk_ldv(fi + (size_t)a * Nvp + k0, fv[a]);
#pragma unroll
            for (int v = 0; v < V; ++v) Nn[a][v] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < AVS_MAXS; ++q) {
            if (q >= ns) break;
            const float* Fq = P.FX + (size_t)fs[q] * cs + k0;
            const float g = sg[q];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                float t[V];
                rk_ldv(Fq + (size_t)a * Nvp, t);
#pragma unroll
                for (int v = 0; v < V; ++v) Nn[a][v] += g * t[v];
            }
        }
        float out[NA][V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float gv[NA];
            rk_eval<D, float>(cp.eq, x[v], gv);
            const bool real = k0 + v < Nv;
#pragma unroll
            for (int a = 0; a < NA; ++a) out[a][v] = real ? (fv[a][v] * u0 + gv[a] * u1 - Nn[a][v] * u2) * u3 : 0.0f;
            float c[D];
#pragma unroll
            for (int d = 0; d < D; ++d) c[d] = x[v][d] - Vn[d];
            rk_raw_acc<D>(acc, c, wv[v] * out[0][v], D == 2 ? wv[v] * out[1][v] : 0.0f, wv[v] * out[NA - 1][v]);
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) rk_stv(fo + (size_t)a * Nvp + k0, out[a]);
    }
    // rows are padded to a multiple of 32 nodes and every thread's k0 is a
    // multiple of V, so the loop above wrote every node below the first k0 >= Nv;
    // the pad nodes from there to Nvp are zeroed here
    for (int k = ((Nv + V - 1) / V) * V + tid; k < Nvp; k += RK_NT)
#pragma unroll
        for (int a = 0; a < NA; ++a) fo[(size_t)a * Nvp + k] = 0.0f;
    block_sum_t<NR, RK_NT>(acc, sw, red);
    if (tid < NR) mom[(size_t)i * NR + tid] = red[tid];
}

// W (and the total heat flux q_t + q_r) of every cell.
template <int D, typename T>
__global__ void __launch_bounds__(RK_NT) rk_moments(int Nv, int Nvp, const T* __restrict__ f,
                                                    const double* __restrict__ xi, const double* __restrict__ w,
                                                    double* Wout, double* qout)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3;
    __shared__ double sred[(RK_NT / 32) * 6], sout[6];
    const int i = blockIdx.x;
    double W[NW], qt[3], qr[3];
    rk_cell_mom<D, T>(f + (size_t)i * NA * Nvp, Nv, Nvp, xi, w, W, qout ? qt : nullptr, qr, sred, sout);
    if (threadIdx.x == 0) {
        if (Wout)
            for (int m = 0; m < NW; ++m) Wout[(size_t)i * NW + m] = W[m];
        if (qout)
            for (int d = 0; d < D; ++d) qout[(size_t)i * D + d] = qt[d] + qr[d];
    }
}

// Conservation correction (Sec. 3.3, reading R30): f <- f + g^M(W) - g^M(W')
// with g^M = (g^eq(T_t), (3 - D) R T_t g^eq(T_t), R T_r g^eq(T_t)), `iters`
// times; the largest remaining relative gap into *gap_key.
template <int D, typename T>
__global__ void __launch_bounds__(RK_NT) rk_correct(int Nv, int Nvp, T* f, const double* __restrict__ xi,
                                                    const double* __restrict__ w, const float* __restrict__ xif,
                                                    const float* __restrict__ wf, const double* __restrict__ Wt,
                                                    RkGas g, int iters, unsigned long long* gap_key)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3, NR = RkNR<D>::v;
    __shared__ double sred[(RK_NT / 32) * NR], sout[NR];
    __shared__ RkEq<T> ea, eb;
    const int i = blockIdx.x;
    T* fi = f + (size_t)i * NA * Nvp;
    const double* Wi = Wt + (size_t)i * NW;
    g.iz = 0.0;
    const double z[3] = {0, 0, 0};
    double rho, U[3], RTt, RTr, RT;
    rk_prim<D>(Wi, rho, U, RTt, RTr, RT);
    if (threadIdx.x == 0) ea = rk_make<D, T>(g, rho, U, RTt, RTr, z, z);
    // mixed form: the moments as FP32 raw sums about V = U(W~) with an FP64
    // combine (the monatomic correction's scheme), the nodes in FP32
    float V[3];
    rk_vref<D>(Wi, V);
    const double Vd[3] = {V[0], V[1], V[2]};
    for (int it = 0; it <= iters; ++it) {
        double Wp[NW];
        if constexpr (sizeof(T) == 4) {
            float acc[NR];
#pragma unroll
            for (int m = 0; m < NR; ++m) acc[m] = 0.0f;
            for (int k = threadIdx.x; k < Nv; k += RK_NT) {
                float c[D];
#pragma unroll
                for (int d = 0; d < D; ++d) c[d] = xif[(size_t)k * D + d] - V[d];
                const float wk = wf[k];
                rk_raw_acc<D>(acc, c, wk * fi[k], D == 2 ? wk * fi[Nvp + k] : 0.0f, wk * fi[(size_t)(NA - 1) * Nvp + k]);
            }
            block_sum_t<NR, RK_NT>(acc, sred, sout);
            if (threadIdx.x == 0) {
                double qd[3], rd[3];
                rk_from_raw<D>(sout, Vd, Wp, qd, rd);
            }
        } else {
            rk_cell_mom<D, T>(fi, Nv, Nvp, xi, w, Wp, nullptr, nullptr, sred, sout);
        }
        if (it == iters) {
            if (threadIdx.x == 0) {
                double mref = 0.0;
                for (int d = 0; d < D; ++d) mref += Wi[1 + d] * Wi[1 + d];
                mref = sqrt(mref) + rho * sqrt(2.0 * RT);
                double e = fabs(Wp[0] - Wi[0]) / fabs(Wi[0]);
                for (int d = 0; d < D; ++d) e = fmax(e, fabs(Wp[1 + d] - Wi[1 + d]) / mref);
                for (int c = D + 1; c < NW; ++c) e = fmax(e, fabs(Wp[c] - Wi[c]) / fabs(Wi[D + 1]));
                if (e != e) e = INFINITY;
                atomicMax(gap_key, dkey(e));
            }
            break;
        }
        if (threadIdx.x == 0) {
            double rp, Up[3], RTtp, RTrp, RTp;
            rk_prim<D>(Wp, rp, Up, RTtp, RTrp, RTp);
            eb = rk_make<D, T>(g, rp, Up, RTtp, RTrp, z, z);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < Nv; k += RK_NT) {
            T xt[D];
#pragma unroll
            for (int d = 0; d < D; ++d) xt[d] = sizeof(T) == 4 ? (T)xif[(size_t)k * D + d] : (T)xi[(size_t)k * D + d];
            T va[NA], vb[NA];
            rk_eval<D, T>(ea, xt, va);
            rk_eval<D, T>(eb, xt, vb);
#pragma unroll
            for (int a = 0; a < NA; ++a) fi[(size_t)a * Nvp + k] += va[a] - vb[a];
        }
        __syncthreads();
    }
}

// conserved -> primitive rho, U, T_t, T_r (the initial-field layout)
template <int D>
__global__ void rk_cons_to_prim(int Nc, const double* __restrict__ Wc, double R, double* Wp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    constexpr int NW = D + 3;
    double rho, U[3], RTt, RTr, RT;
    rk_prim<D>(Wc + (size_t)i * NW, rho, U, RTt, RTr, RT);
    double* P = Wp + (size_t)i * NW;
    P[0] = rho;
    for (int d = 0; d < D; ++d) P[1 + d] = U[d];
    P[D + 1] = RTt / R;
    P[D + 2] = RTr / R;
}

// ---------------------------------------------------------------- implicit step
// IUGKS for the Rykov model (Sec. 2.3.1): the face stage of the explicit step,
// then Eq. (SGS_w) for rho, rho U, rho E and Eq. (SGS_wrot) for rho E_rot by
// symmetric Gauss-Seidel over the cell colouring (one cooperative launch,
// bounded grid barrier between colour passes), then Eq. (SGS_phi) for G, H,
// R.  The same structure as the monatomic implicit step; readings R31-R32.

// Euler flux of a diatomic gas: p = rho R T (equilibrium T of the total
// energy), rho E_rot carried with the flow.
template <int D, typename A>
__device__ __forceinline__ void rk_euler_flux(const A* W, const A* n, A* G)
{
    const A rho = W[0];
    A m2 = A(0), un = A(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        m2 += W[1 + d] * W[1 + d];
        un += (W[1 + d] / rho) * n[d];
    }
    const A p = rho * ((W[D + 1] - A(0.5) * m2 / rho) / (A(2.5) * rho));
    G[0] = rho * un;
#pragma unroll
    for (int d = 0; d < D; ++d) G[1 + d] = W[1 + d] * un + p * n[d];
    G[D + 1] = (W[D + 1] + p) * un;
    G[D + 2] = W[D + 2] * un;
}

template <typename A>
struct RkImpSlot {
    A n[3];
    A nhA;
    A hr;
    A Gn[6];
    int j;
};
static_assert(sizeof(RkImpSlot<double>) <= AVS_IMPSLOT_BYTES, "slot record");

template <typename A>
struct RkImpP {
    int Nc;
    double dt;
    RkGas g;
    const int* slot;
    const unsigned char* nslot;
    const int* faceL;
    const int* faceR;
    const double* An;
    const double* rL;
    const double* rR;
    const double* vol;
    const double* AF;
    const double* Wn;        // W^n [cell][NW]
    double* Wt;              // W~ [cell][NW]
    A* dWa;                  // dW [cell][NW]
    A* Wta;                  // W~ in A [cell][NW]; aliases Wt when A is double
    A* rhs;                  // [q][NW]
    A* dg;                   // [q]
    RkImpSlot<A>* co;        // [q][MAXS]
    unsigned char* nint;     // [q]
    const int* clist;
    int* err;
};

template <int D, typename A>
__global__ void rk_imp_setup(RkImpP<A> P)
{
    constexpr int NW = D + 3;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P.Nc) return;
    const int i = P.clist[q];
    const int ns = P.nslot[i];
    const double* Wi = P.Wn + (size_t)i * NW;
    for (int c = 0; c < NW; ++c) {
        double acc = 0.0;
        for (int s = 0; s < ns; ++s) {
            const int sl = P.slot[i * AVS_MAXS + s];
            const double a = P.AF[(size_t)(sl >> 1) * NW + c];
            acc += (sl & 1) ? -a : a;
        }
        P.rhs[(size_t)q * NW + c] = (A)(-acc);
        P.dWa[(size_t)i * NW + c] = A(0);
        P.Wt[(size_t)i * NW + c] = Wi[c];
        P.Wta[(size_t)i * NW + c] = (A)Wi[c];
    }
    double dg = P.vol[i] / P.dt;
    int nint = 0;
    for (int s = 0; s < ns; ++s) {
        const int sl = P.slot[i * AVS_MAXS + s];
        const int f = sl >> 1;
        const double sgn = (sl & 1) ? -1.0 : 1.0;
        const int L = P.faceL[f], R = P.faceR[f];
        const double* An = P.An + (size_t)f * D;
        double Aa = 0.0;
        for (int d = 0; d < D; ++d) Aa += An[d] * An[d];
        Aa = sqrt(Aa);
        double n[3] = {0, 0, 0}, dl = 0.0;
        for (int d = 0; d < D; ++d) n[d] = An[d] / Aa;
        for (int d = 0; d < D; ++d) {
            const double e = R >= 0 ? P.rL[(size_t)f * D + d] - P.rR[(size_t)f * D + d] : 2.0 * P.rL[(size_t)f * D + d];
            dl += e * e;
        }
        dl = sqrt(dl);
        // radius |U.n| + a + 2 mu / (rho dl): a = sqrt(7/5 R T), mu at the mean T_t (R31)
        double rl, Ul[3], tl, ql, RTl, rr, Ur[3], tr, qr2, RTr;
        rk_prim<D>(P.Wn + (size_t)L * NW, rl, Ul, tl, ql, RTl);
        rk_prim<D>(P.Wn + (size_t)(R >= 0 ? R : L) * NW, rr, Ur, tr, qr2, RTr);
        const double rho = 0.5 * (rl + rr), RT = 0.5 * (RTl + RTr), RTt = 0.5 * (tl + tr);
        double un = 0.0;
        for (int d = 0; d < D; ++d) un += 0.5 * (Ul[d] + Ur[d]) * n[d];
        const double mu = P.g.mu_ref * pow(RTt / P.g.R / P.g.T_ref, P.g.omega);
        const double r = Aa * (fabs(un) + sqrt(7.0 / 5.0 * RT) + 2.0 * mu / (rho * dl));
        dg += 0.5 * r;
        const int j = (sl & 1) ? L : R;
        if (j >= 0) {
            RkImpSlot<A> sc;
            for (int d = 0; d < 3; ++d) sc.n[d] = d < D ? (A)(sgn * An[d] / Aa) : A(0);
            sc.nhA = (A)(-0.5 * Aa);
            sc.hr = (A)(0.5 * r);
            A Wj[NW];
            for (int c = 0; c < NW; ++c) Wj[c] = (A)P.Wn[(size_t)j * NW + c];
            rk_euler_flux<D, A>(Wj, sc.n, sc.Gn);
            for (int c = NW; c < 6; ++c) sc.Gn[c] = A(0);
            sc.j = j;
            P.co[(size_t)q * AVS_MAXS + nint++] = sc;
        }
    }
    P.dg[q] = (A)dg;
    P.nint[q] = (unsigned char)nint;
}

// One cell of a macroscopic sweep, with the rotational source of Eq.
// (SGS_wrot) from the cell's current W~ (reading R32).
template <int D, typename A>
__device__ __forceinline__ void rk_imp_cell(const RkImpP<A>& P, int q)
{
    constexpr int NW = D + 3;
    const int i = P.clist[q];
    const int n = P.nint[q];
    A rhs[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) rhs[c] = P.rhs[(size_t)q * NW + c];
    for (int s = 0; s < n; ++s) {
        const RkImpSlot<A> sc = P.co[(size_t)q * AVS_MAXS + s];
        A Wj[NW], dWj[NW], G[NW];
#pragma unroll
        for (int c = 0; c < NW; ++c) {
            Wj[c] = __ldcg(P.Wta + (size_t)sc.j * NW + c);
            dWj[c] = __ldcg(P.dWa + (size_t)sc.j * NW + c);
        }
        rk_euler_flux<D, A>(Wj, sc.n, G);
#pragma unroll
        for (int c = 0; c < NW; ++c) rhs[c] += sc.nhA * (G[c] - sc.Gn[c]) + sc.hr * dWj[c];
    }
    const A dg = P.dg[q];
    A dgr = dg;
    {
        A W[NW];
#pragma unroll
        for (int c = 0; c < NW; ++c) W[c] = __ldcg(P.Wta + (size_t)i * NW + c);
        const A rho = W[0];
        A m2 = A(0);
#pragma unroll
        for (int d = 0; d < D; ++d) m2 += W[1 + d] * W[1 + d];
        const A eint = W[D + 1] - A(0.5) * m2 / rho;
        const A RT = eint / (A(2.5) * rho);
        const A RTt = (eint - W[D + 2]) / (A(1.5) * rho);
        if (!(rho > A(0)) || !(RTt > A(0)) || !(RT > A(0))) atomicOr(P.err, 1);
        const A T = RTt / (A)P.g.R;
        const A mu = (A)P.g.mu_ref * powa(T / (A)P.g.T_ref, (A)P.g.omega);
        const A tau = mu / (rho * RTt);
        const A V = (A)P.vol[i], Z = (A)P.g.Z;
        rhs[D + 2] += V * (rho * RT - (A)P.Wn[(size_t)i * NW + D + 2]) / (Z * tau);
        dgr = dg + V / (Z * tau);
    }
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        const A d = rhs[c] / (c == D + 2 ? dgr : dg);
        const double wt = P.Wn[(size_t)i * NW + c] + (double)d;
        __stcg(P.dWa + (size_t)i * NW + c, d);
        if constexpr (sizeof(A) == sizeof(double)) {
            __stcg(P.Wt + (size_t)i * NW + c, wt);
        } else {
            P.Wt[(size_t)i * NW + c] = wt;
            __stcg(P.Wta + (size_t)i * NW + c, (A)wt);
        }
    }
}

// All colour passes of the macroscopic solve in one cooperative launch.
// Unlike the monatomic sweep, a colour that follows itself is not skipped:
// the rotational source reads the cell's own W~, which the first of the two
// passes changes.
template <int D, typename A, int NT>
__global__ void __launch_bounds__(NT) rk_imp_macro(RkImpP<A> P, int k_macro, int ncolor,
                                                   const int* __restrict__ cstart, unsigned* bar)
{
    const unsigned nb = gridDim.x;
    unsigned gen = 0;
    bool first = true;
    for (int it = 0; it < k_macro; ++it)
        for (int dir = 0; dir < 2; ++dir)
            for (int qq = 0; qq < ncolor; ++qq) {
                const int col = dir == 0 ? qq : ncolor - 1 - qq;
                if (!first && !grid_sync_bounded(bar, ++gen * nb, P.err)) return;
                first = false;
                const int c1 = cstart[col + 1];
                for (int q = cstart[col] + blockIdx.x * NT + threadIdx.x; q < c1; q += nb * NT)
                    rk_imp_cell<D, A>(P, q);
            }
}
// rk_imp_res for the mixed form: the raw moments of f^n and the residual
// RK_VC nodes per thread in vector loads (the cell kernel's layout), the
// state of W~ by thread 0 (FP64 W~, FP32 tau~ and equilibrium).
template <int D>
__global__ void __launch_bounds__(RK_NT, 7) rk_imp_res32(RkP<float> P, const float* __restrict__ xif,
                                                         const float* __restrict__ wf, double* u0)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3, NR = RkNR<D>::v, V = RK_VC;
    __shared__ double sw[(RK_NT / 32) * NR], red[NR];
    __shared__ RkEq<float> eq;
    __shared__ float ctau, cvol, cV[3];
    __shared__ double Vd[3];
    __shared__ int fs[AVS_MAXS];
    __shared__ float sg[AVS_MAXS];
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int ns = P.nslot[i];
    const int Nv = P.Nv, Nvp = P.Nvp;
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        fs[tid] = sl >> 1;
        sg[tid] = (sl & 1) ? -1.0f : 1.0f;
    }
    if (tid == 32) {
        rk_vref<D>(P.Win + (size_t)i * NW, cV);
        for (int d = 0; d < 3; ++d) Vd[d] = cV[d];
        cvol = (float)P.vol[i];
    }
    __syncthreads();
    const size_t cs = (size_t)NA * Nvp;
    const float* fi = P.f + (size_t)i * cs;
    float Vr[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vr[d] = cV[d];
    float acc[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) acc[m] = 0.0f;
    for (int k0 = tid * V; k0 < Nv; k0 += RK_NT * V) {
        float x[V][D], wv[V], fv[NA][V];
        rk_ld_nodes<D>(xif, wf, k0, x, wv);
#pragma unroll
        for (int a = 0; a < NA; ++a) rk_ldv(fi + (size_t)a * Nvp + k0, fv[a]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float c[D];
#pragma unroll
            for (int d = 0; d < D; ++d) c[d] = x[v][d] - Vr[d];
            rk_raw_acc<D>(acc, c, wv[v] * fv[0][v], D == 2 ? wv[v] * fv[1][v] : 0.0f, wv[v] * fv[NA - 1][v]);
        }
    }
    block_sum_t<NR, RK_NT>(acc, sw, red);
    if (tid == 0) {
        float rn, Un[3], etn, r0n, qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
        rk_state_raw32<D>(red, Vd, rn, Un, etn, r0n, qt, qr);
        double rho, U[3], RTt, RTr, RT;
        rk_prim<D>(P.Wout + (size_t)i * NW, rho, U, RTt, RTr, RT);
        if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
        const float tau = rk_tau32(P.g, (float)rho, (float)RTt);
        float Uf[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) Uf[d] = (float)U[d];
        eq = rk_make32<D>(P.g, (float)rho, Uf, (float)RTt, (float)RTr, qt, qr);
        ctau = tau;
        u0[i] = P.vol[i] / P.dt + P.vol[i] / (double)tau;
    }
    __syncthreads();
    const float Vc = cvol, vit = cvol / ctau;
    float* ro = P.fout + (size_t)i * cs;
    for (int k0 = tid * V; k0 < Nv; k0 += RK_NT * V) {
        float x[V][D], wv[V], fv[NA][V], Nn[NA][V];
        rk_ld_nodes<D>(xif, wf, k0, x, wv);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            rk_ldv(fi + (size_t)a * Nvp + k0, fv[a]);
#pragma unroll
            for (int v = 0; v < V; ++v) Nn[a][v] = 0.0f;
        }
#pragma unroll
        for (int q = 0; q < AVS_MAXS; ++q) {
            if (q >= ns) break;
            const float* Fq = P.FX + (size_t)fs[q] * cs + k0;
            const float g = sg[q];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                float t[V];
                rk_ldv(Fq + (size_t)a * Nvp, t);
#pragma unroll
                for (int v = 0; v < V; ++v) Nn[a][v] += g * t[v];
            }
        }
        float out[NA][V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float gv[NA];
            rk_eval<D, float>(eq, x[v], gv);
            const bool real = k0 + v < Nv;
#pragma unroll
            for (int a = 0; a < NA; ++a) out[a][v] = real ? (gv[a] - fv[a][v]) * vit - Nn[a][v] : 0.0f;
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) rk_stv(ro + (size_t)a * Nvp + k0, out[a]);
    }
    for (int k = ((Nv + V - 1) / V) * V + tid; k < Nvp; k += RK_NT)
#pragma unroll
        for (int a = 0; a < NA; ++a) ro[(size_t)a * Nvp + k] = 0.0f;
    (void)Vc;
}

// Per cell: Rykov state of W~ with the lagged q_t, q_r of f^n, and the
// microscopic residual Res = V (g~ - phi^n) / tau~ - N of every array (written
// over the f^{n+1} buffer); u0[i] = V/dt + V/tau~ for the sweeps.
template <int D, typename T>
__global__ void __launch_bounds__(RK_NT) rk_imp_res(RkP<T> P, const T* __restrict__ xiT,
                                                    const T* __restrict__ wT, double* u0)
{
    static_assert(sizeof(T) == 8, "the mixed form uses rk_imp_res32");
    constexpr int NA = RkNA<D>::v, NW = D + 3;
    __shared__ double sred[(RK_NT / 32) * RkNR<3>::v], sout[RkNR<3>::v];
    __shared__ RkEq<T> eq;
    __shared__ double tau_s;
    __shared__ int fs[AVS_MAXS];
    __shared__ T sg[AVS_MAXS];
    const int i = blockIdx.x;
    const int ns = P.nslot[i];
    const int Nv = P.Nv, Nvp = P.Nvp;
    if (threadIdx.x < ns) {
        const int sl = P.slot[i * AVS_MAXS + threadIdx.x];
        fs[threadIdx.x] = sl >> 1;
        sg[threadIdx.x] = (sl & 1) ? T(-1) : T(1);
    }
    const size_t cs = (size_t)NA * Nvp;
    const T* fi = P.f + (size_t)i * cs;
    double qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
    {
        double Wn[NW];
        rk_cell_mom<D, T>(fi, Nv, Nvp, P.xi, P.w, Wn, qt, qr, sred, sout);
        if (threadIdx.x == 0) {
            double rho, U[3], RTt, RTr, RT;
            rk_prim<D>(P.Wout + (size_t)i * NW, rho, U, RTt, RTr, RT);
            if (!(rho > 0.0) || !(RTt > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
            const double tau = rk_tau(P.g, rho, RTt);
            eq = rk_make<D, T>(P.g, rho, U, RTt, RTr, qt, qr);
            tau_s = tau;
            u0[i] = P.vol[i] / P.dt + P.vol[i] / tau;
        }
    }
    __syncthreads();
    const T tau = (T)tau_s, Vc = (T)P.vol[i];
    T* ro = P.fout + (size_t)i * cs;
    for (int k = threadIdx.x; k < Nvp; k += RK_NT) {
        if (k >= Nv) {
#pragma unroll
            for (int a = 0; a < NA; ++a) ro[(size_t)a * Nvp + k] = T(0);
            continue;
        }
        T xt[D];
#pragma unroll
        for (int d = 0; d < D; ++d) xt[d] = xiT[(size_t)k * D + d];
        T gv[NA];
        rk_eval<D, T>(eq, xt, gv);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            T N = T(0);
            for (int q = 0; q < ns; ++q) N += sg[q] * P.FX[((size_t)fs[q] * NA + a) * Nvp + k];
            ro[(size_t)a * Nvp + k] = Vc * (gv[a] - fi[(size_t)a * Nvp + k]) / tau - N;
        }
    }
}

// One colour of a microscopic sweep (Eq. SGS_phi), every node and array:
// dphi_i = (Res_i - sum_{xi.n<0} (xi.n) dphi_j) / (u0_i + sum_{xi.n>=0} xi.n).
template <int D, typename T>
__global__ void __launch_bounds__(RK_NT) rk_imp_micro(int Nv, int Nvp, const T* __restrict__ res, T* dphi,
                                                      const double* __restrict__ u0, const T* __restrict__ xiT,
                                                      const double* __restrict__ xid, const double* __restrict__ Ad,
                                                      const T* __restrict__ An, const int* __restrict__ slot,
                                                      const unsigned char* __restrict__ nslot,
                                                      const int* __restrict__ faceL, const int* __restrict__ faceR,
                                                      const int* __restrict__ clist, int c0)
{
    static_assert(sizeof(T) == 8, "the mixed form uses rk_imp_micro32");
    constexpr int NA = RkNA<D>::v;
    __shared__ double sAd[AVS_MAXS][3];
    __shared__ int snb[AVS_MAXS];
    const int i = clist[c0 + blockIdx.x];
    const int ns = nslot[i];
    if (threadIdx.x < ns) {
        const int sl = slot[i * AVS_MAXS + threadIdx.x];
        const int f = sl >> 1;
        for (int d = 0; d < D; ++d) sAd[threadIdx.x][d] = (sl & 1) ? -Ad[(size_t)f * D + d] : Ad[(size_t)f * D + d];
        snb[threadIdx.x] = (sl & 1) ? faceL[f] : faceR[f];
    }
    __syncthreads();
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= Nvp) return;
    if (k >= Nv) {
        for (int a = 0; a < NA; ++a) dphi[((size_t)i * NA + a) * Nvp + k] = T(0);
        return;
    }
    // xi . n per slot in FP64 without contraction (the oracle's upwind split)
    T sn[AVS_MAXS];
    T out = T(0);
    for (int s = 0; s < ns; ++s) {
        double xd[3] = {0, 0, 0};
        for (int d = 0; d < D; ++d) xd[d] = xid[(size_t)k * D + d];
        const T v = (T)dot_rn<D>(xd, sAd[s]);
        sn[s] = v;
        if (v >= T(0)) out += v;
    }
    const T dg = (T)u0[i] + out;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        T acc = res[((size_t)i * NA + a) * Nvp + k];
        for (int s = 0; s < ns; ++s)
            if (snb[s] >= 0 && sn[s] < T(0)) acc -= sn[s] * dphi[((size_t)snb[s] * NA + a) * Nvp + k];
        dphi[((size_t)i * NA + a) * Nvp + k] = acc / dg;
    }
}

// One colour of a microscopic sweep in the mixed form: as rk_imp_micro, four
// nodes per thread in 16-byte vectors; a neighbour's dphi row is read only
// when one of the four nodes is downwind of it.
template <int D>
__global__ void __launch_bounds__(RK_NT) rk_imp_micro32(int Nv, int Nvp, const float* __restrict__ res, float* dphi,
                                                        const double* __restrict__ u0, const float* __restrict__ xif,
                                                        const float* __restrict__ An, const int* __restrict__ slot,
                                                        const unsigned char* __restrict__ nslot,
                                                        const int* __restrict__ faceL, const int* __restrict__ faceR,
                                                        const int* __restrict__ clist, int c0)
{
    constexpr int NA = RkNA<D>::v, V = 4;
    __shared__ float sA[AVS_MAXS][D];
    __shared__ int snb[AVS_MAXS];
    __shared__ float su0;
    const int tid = threadIdx.x;
    const int i = clist[c0 + blockIdx.x];
    const int ns = nslot[i];
    if (tid < ns) {
        const int sl = slot[i * AVS_MAXS + tid];
        const int f = sl >> 1;
#pragma unroll
        for (int d = 0; d < D; ++d) sA[tid][d] = (sl & 1) ? -An[(size_t)f * D + d] : An[(size_t)f * D + d];
        snb[tid] = (sl & 1) ? faceL[f] : faceR[f];
    }
    if (tid == 32) su0 = (float)u0[i];
    __syncthreads();
    const int k0 = (blockIdx.y * RK_NT + tid) * V;
    if (k0 >= Nv) return;                          // pad nodes keep the zero of the initial dphi
    float x[V][D];
    {
        float t[V * D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(xif + (size_t)k0 * D) + j);
            t[4 * j] = q.x;
            t[4 * j + 1] = q.y;
            t[4 * j + 2] = q.z;
            t[4 * j + 3] = q.w;
        }
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int d = 0; d < D; ++d) x[v][d] = t[v * D + d];
    }
    float sn[AVS_MAXS][V], idg[V];
#pragma unroll
    for (int v = 0; v < V; ++v) idg[v] = 0.0f;
#pragma unroll
    for (int s = 0; s < AVS_MAXS; ++s) {
        if (s >= ns) break;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float p = 0.0f;
#pragma unroll
            for (int d = 0; d < D; ++d) p += x[v][d] * sA[s][d];
            sn[s][v] = p;
            if (p >= 0.0f) idg[v] += p;
        }
    }
    const float u = su0;
#pragma unroll
    for (int v = 0; v < V; ++v) idg[v] = 1.0f / (u + idg[v]);
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const float4 r4 = __ldcg(reinterpret_cast<const float4*>(res + ((size_t)i * NA + a) * Nvp + k0));
        float acc[V] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
        for (int s = 0; s < AVS_MAXS; ++s) {
            if (s >= ns) break;
            const int j = snb[s];
            bool in = false;
#pragma unroll
            for (int v = 0; v < V; ++v) in |= sn[s][v] < 0.0f;
            if (j < 0 || !in) continue;
            const float4 t4 = __ldcg(reinterpret_cast<const float4*>(dphi + ((size_t)j * NA + a) * Nvp + k0));
            const float t[V] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (sn[s][v] < 0.0f) acc[v] -= sn[s][v] * t[v];
        }
        float o[V];
#pragma unroll
        for (int v = 0; v < V; ++v) o[v] = k0 + v < Nv ? acc[v] * idg[v] : 0.0f;
        *reinterpret_cast<float4*>(dphi + ((size_t)i * NA + a) * Nvp + k0) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// f^{n+1} = f^n + dphi (pad nodes zero)
template <typename T>
__global__ void rk_imp_finish(int Nv, int Nvp, const T* __restrict__ fin, const T* __restrict__ dphi, T* fout)
{
    const int r = blockIdx.x;
    for (int k = blockIdx.y * blockDim.x + threadIdx.x; k < Nvp; k += gridDim.y * blockDim.x)
        fout[(size_t)r * Nvp + k] = k < Nv ? fin[(size_t)r * Nvp + k] + dphi[(size_t)r * Nvp + k] : T(0);
}

RkGas rk_gas(const avs_ctx* c)
{
    RkGas g;
    g.R = c->cfg.R;
    g.mu_ref = c->mu_ref;
    g.T_ref = c->cfg.T_ref;
    g.omega = c->cfg.omega;
    g.Z = c->cfg.Zrot;
    g.iz = 1.0 / c->cfg.Zrot;
    g.om0 = AVS_RYKOV_OMEGA0;
    g.om1 = AVS_RYKOV_OMEGA1;
    g.dl = AVS_RYKOV_DELTA;
    return g;
}

cudaError_t ensure_bytes(void** p, size_t* have, size_t need)
{
    if (*have >= need) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, need);
    if (e == cudaSuccess) *have = need;
    return e;
}

// Gradient and face kernels of a step: fills P and launches them.
template <int D, typename T>
cudaError_t rk_face_stage(avs_ctx* c, const void* fin, const double* Win, double dt, RkP<T>& P)
{
    constexpr int NA = RkNA<D>::v;
    const size_t rows = (size_t)std::max(c->fcap, c->Nvp);
    const bool grad = c->cfg.limiter != 0;
    cudaError_t e;
    if (grad) {
        e = ensure_bytes(&c->grad, &c->grad_bytes, (size_t)c->Nc * NA * D * rows * sizeof(T));
        if (e != cudaSuccess) return e;
    }
    // the face flux, and in the implicit step afterwards the per-cell dphi
    e = ensure_bytes(&c->flux, &c->flux_bytes, (size_t)std::max(c->Nf, c->Nc) * NA * rows * sizeof(T));
    if (e != cudaSuccess) return e;
    P.Nv = c->Nv;
    P.Nvp = c->Nvp;
    P.Nc = c->Nc;
    P.limiter = c->cfg.limiter;
    P.dt = dt;
    P.h = 0.5 * dt;
    P.g = rk_gas(c);
    P.order = c->forder;
    P.faceL = c->faceL;
    P.faceR = c->faceR;
    P.An = c->An_d;
    P.rL = c->rL_d;
    P.rR = c->rR_d;
    P.bc = c->bc;
    P.xi = c->xi_d;
    P.w = c->w_d;
    P.vol = c->vol;
    P.slot = c->slot;
    P.nslot = c->nslot;
    P.f = (const T*)fin;
    P.G = grad ? (const T*)c->grad : nullptr;
    P.FX = (T*)c->flux;
    P.AF = c->AFf;
    P.Win = Win;
    P.Wout = nullptr;
    P.fout = nullptr;
    P.err = c->dev_err;
    if (grad) launch_grad_rykov(c, fin);     // the monatomic gradient kernel over NA arrays
    if constexpr (sizeof(T) == 4)
        rk_face32<D><<<c->Nf, RK_NT, 0, c->stream>>>(P, c->xi_f, c->w_f, c->An_f, c->rL_f, c->rR_f);
    else
        rk_face<D, T><<<c->Nf, RK_NT, 0, c->stream>>>(P);
    c->launches += 1;
    return cudaGetLastError();
}

template <int D, typename T>
cudaError_t rk_step_t(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt)
{
    RkP<T> P;
    cudaError_t e = rk_face_stage<D, T>(c, fin, Win, dt, P);
    if (e != cudaSuccess) return e;
    P.Wout = Wout;
    P.fout = (T*)fout;
    if constexpr (sizeof(T) == 4) {
        RkCellPar* par = reinterpret_cast<RkCellPar*>(c->cpar);
        if (!c->mom_valid) {
            rk_raw_moments32<D><<<c->Nc, RK_NT, 0, c->stream>>>(P, c->xi_f, c->w_f, c->cmom);
            c->launches += 1;
        }
        rk_cell_state32<D><<<(c->Nc + 127) / 128, 128, 0, c->stream>>>(P, c->cmom, par);
        rk_cell32<D><<<c->Nc, RK_NT, 0, c->stream>>>(P, c->xi_f, c->w_f, c->cmom, par);
        c->launches += 2;
        c->mom_valid = 1;      // the raw moments of fout about V(Wout) are in cmom
    } else {
        rk_cell<D, T><<<c->Nc, RK_NT, 0, c->stream>>>(P);
        c->launches += 1;
        c->mom_valid = 0;
    }
    return cudaGetLastError();
}

template <int D, typename T>
cudaError_t rk_step_implicit_t(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt,
                               int k_macro, int k_micro)
{
    constexpr int NA = RkNA<D>::v;
    const bool f32 = sizeof(T) == 4;
    RkP<T> P;
    cudaError_t e = rk_face_stage<D, T>(c, fin, Win, dt, P);
    if (e != cudaSuccess) return e;
    // ---- macroscopic system, Eqs. (SGS_w), (SGS_wrot)
    using A = T;
    RkImpP<A> I;
    I.Nc = c->Nc;
    I.dt = dt;
    I.g = P.g;
    I.slot = c->slot;
    I.nslot = c->nslot;
    I.faceL = c->faceL;
    I.faceR = c->faceR;
    I.An = c->An_d;
    I.rL = c->rL_d;
    I.rR = c->rR_d;
    I.vol = c->vol;
    I.AF = c->AFf;
    I.Wn = Win;
    I.Wt = Wout;
    I.dWa = (A*)c->imp_dW;
    I.Wta = f32 ? (A*)c->imp_Wta : (A*)Wout;
    I.rhs = (A*)c->imp_rhs0;
    I.dg = (A*)c->imp_diag;
    I.co = (RkImpSlot<A>*)c->imp_co;
    I.nint = c->imp_nint;
    I.clist = c->clist;
    I.err = c->dev_err;
    const int cb = (c->Nc + 127) / 128;
    rk_imp_setup<D, A><<<cb, 128, 0, c->stream>>>(I);
    c->launches += 1;
    const int nc = c->ncolor;
    if (k_macro > 0) {
        constexpr int NTM = 128;
        int maxcol = 0;
        for (int k = 0; k < nc; ++k) maxcol = std::max(maxcol, c->cstart[k + 1] - c->cstart[k]);
        int dev = 0, nsm = 0, occ = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rk_imp_macro<D, A, NTM>, NTM, 0);
        if (e != cudaSuccess) return e;
        const int nblk = std::max(1, std::min(nsm * std::max(occ, 1), (maxcol + NTM - 1) / NTM));
        e = cudaMemsetAsync(c->imp_bar, 0, sizeof(unsigned), c->stream);
        if (e != cudaSuccess) return e;
        int km = k_macro, ncol = nc;
        const int* cs = c->cstart_d;
        unsigned* bar = c->imp_bar;
        void* args[] = {&I, &km, &ncol, &cs, &bar};
        e = cudaLaunchCooperativeKernel((const void*)rk_imp_macro<D, A, NTM>, dim3(nblk), dim3(NTM), args, 0,
                                        c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 1;
    }
    // ---- microscopic system, Eq. (SGS_phi)
    P.Wout = Wout;                      // W~
    P.fout = (T*)fout;                  // holds the residual until the finish
    double* u0 = c->imp_diag;           // the macroscopic diagonal is no longer needed
    if constexpr (sizeof(T) == 4)
        rk_imp_res32<D><<<c->Nc, RK_NT, 0, c->stream>>>(P, c->xi_f, c->w_f, u0);
    else
        rk_imp_res<D, T><<<c->Nc, RK_NT, 0, c->stream>>>(P, c->xi_d, c->w_d, u0);
    c->launches += 1;
    T* dphi = (T*)c->flux;              // the face flux has been used
    e = cudaMemsetAsync(dphi, 0, (size_t)c->Nc * NA * c->Nvp * sizeof(T), c->stream);
    if (e != cudaSuccess) return e;
    const int nyb = (c->Nvp + 127) / 128;
    int prev = -1;
    for (int it = 0; it < k_micro; ++it)
        for (int dir = 0; dir < 2; ++dir)
            for (int q = 0; q < nc; ++q) {
                const int col = dir == 0 ? q : nc - 1 - q;
                if (col == prev) continue;      // same inputs as the pass before: same values
                prev = col;
                const int c0 = c->cstart[col], c1 = c->cstart[col + 1];
                if (c1 <= c0) continue;
                if constexpr (sizeof(T) == 4) {
                    rk_imp_micro32<D><<<dim3(c1 - c0, (c->Nv + RK_NT * 4 - 1) / (RK_NT * 4)), RK_NT, 0, c->stream>>>(
                        c->Nv, c->Nvp, (const float*)fout, (float*)dphi, u0, c->xi_f, c->An_f, c->slot, c->nslot,
                        c->faceL, c->faceR, c->clist, c0);
                    c->launches += 1;
                } else {
                    rk_imp_micro<D, T><<<dim3(c1 - c0, nyb), 128, 0, c->stream>>>(
                        c->Nv, c->Nvp, (const T*)fout, dphi, u0, f32 ? (const T*)c->xi_f : (const T*)c->xi_d,
                        c->xi_d, c->An_d, f32 ? (const T*)c->An_f : (const T*)c->An_d, c->slot, c->nslot, c->faceL,
                        c->faceR, c->clist, c0);
                    c->launches += 1;
                }
            }
    dim3 gf(c->Nc * NA, std::min(8, (c->Nvp + 255) / 256));
    rk_imp_finish<T><<<gf, 256, 0, c->stream>>>(c->Nv, c->Nvp, (const T*)fin, dphi, (T*)fout);
    c->launches += 1;
    c->mom_valid = 0;          // no carried moments of fout
    return cudaGetLastError();
}

}  // namespace

cudaError_t rk_launch_step(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt)
{
    if (c->D == 2)
        return c->mixed ? rk_step_t<2, float>(c, fin, fout, Win, Wout, dt)
                        : rk_step_t<2, double>(c, fin, fout, Win, Wout, dt);
    return c->mixed ? rk_step_t<3, float>(c, fin, fout, Win, Wout, dt)
                    : rk_step_t<3, double>(c, fin, fout, Win, Wout, dt);
}

cudaError_t rk_launch_step_implicit(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout,
                                    double dt, int k_macro, int k_micro)
{
    if (c->D == 2)
        return c->mixed ? rk_step_implicit_t<2, float>(c, fin, fout, Win, Wout, dt, k_macro, k_micro)
                        : rk_step_implicit_t<2, double>(c, fin, fout, Win, Wout, dt, k_macro, k_micro);
    return c->mixed ? rk_step_implicit_t<3, float>(c, fin, fout, Win, Wout, dt, k_macro, k_micro)
                    : rk_step_implicit_t<3, double>(c, fin, fout, Win, Wout, dt, k_macro, k_micro);
}

// W and the total heat flux of every cell in the mixed form: FP32 raw sums
// about the carried velocity (when given) with an FP64 combine, converted by
// the shift formulas (the monatomic moments' scheme; FP64 node sums cost as
// much as the rest of an adaptation).
template <int D>
__global__ void __launch_bounds__(RK_NT) rk_moments32(int Nv, int Nvp, const float* __restrict__ f,
                                                      const float* __restrict__ xif, const float* __restrict__ wf,
                                                      const double* __restrict__ Wref, double* Wout, double* qout)
{
    constexpr int NA = RkNA<D>::v, NW = D + 3, NR = RkNR<D>::v, V = RK_VC;
    __shared__ double sw[(RK_NT / 32) * NR], red[NR];
    __shared__ float cV[3];
    __shared__ double Vd[3];
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    if (tid == 32) {
        cV[0] = cV[1] = cV[2] = 0.0f;
        if (Wref && Wref[(size_t)i * NW] > 0.0) {
            rk_vref<D>(Wref + (size_t)i * NW, cV);
            for (int d = 0; d < 3; ++d)
                if (!isfinite(cV[d])) cV[d] = 0.0f;
        }
        for (int d = 0; d < 3; ++d) Vd[d] = cV[d];
    }
    __syncthreads();
    float Vr[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vr[d] = cV[d];
    const float* fi = f + (size_t)i * NA * Nvp;
    float acc[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) acc[m] = 0.0f;
    for (int k0 = tid * V; k0 < Nv; k0 += RK_NT * V) {
        float x[V][D], wv[V], fv[NA][V];
        rk_ld_nodes<D>(xif, wf, k0, x, wv);
#pragma unroll
        for (int a = 0; a < NA; ++a) rk_ldv(fi + (size_t)a * Nvp + k0, fv[a]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float c[D];
#pragma unroll
            for (int d = 0; d < D; ++d) c[d] = x[v][d] - Vr[d];
            rk_raw_acc<D>(acc, c, wv[v] * fv[0][v], D == 2 ? wv[v] * fv[1][v] : 0.0f, wv[v] * fv[NA - 1][v]);
        }
    }
    block_sum_t<NR, RK_NT>(acc, sw, red);
    if (tid == 0) {
        double W[NW], qt[3] = {0, 0, 0}, qr[3] = {0, 0, 0};
        rk_from_raw<D>(red, Vd, W, qt, qr);
        if (Wout)
            for (int m = 0; m < NW; ++m) Wout[(size_t)i * NW + m] = W[m];
        if (qout)
            for (int d = 0; d < D; ++d) qout[(size_t)i * D + d] = qt[d] + qr[d];
    }
}

cudaError_t rk_launch_moments(avs_ctx* c, const void* f, int f_is_double, int Ncells, int Nvp, double* Wout,
                              double* qout)
{
    const bool dbl = f_is_double || !c->mixed;
    // the carried W as the reference velocity of the sums, unless it is the
    // output (the initial field, whose carried W is being formed)
    const double* Wref = (Ncells == c->Nc && Wout != c->W[c->wcur]) ? c->W[c->wcur] : nullptr;
    if (c->D == 2) {
        if (dbl) rk_moments<2, double><<<Ncells, RK_NT, 0, c->stream>>>(c->Nv, Nvp, (const double*)f, c->xi_d,
                                                                        c->w_d, Wout, qout);
        else rk_moments32<2><<<Ncells, RK_NT, 0, c->stream>>>(c->Nv, Nvp, (const float*)f, c->xi_f, c->w_f, Wref,
                                                              Wout, qout);
    } else {
        if (dbl) rk_moments<3, double><<<Ncells, RK_NT, 0, c->stream>>>(c->Nv, Nvp, (const double*)f, c->xi_d,
                                                                        c->w_d, Wout, qout);
        else rk_moments32<3><<<Ncells, RK_NT, 0, c->stream>>>(c->Nv, Nvp, (const float*)f, c->xi_f, c->w_f, Wref,
                                                              Wout, qout);
    }
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t rk_launch_correct(avs_ctx* c, void* f, const double* Wtarget, int iters)
{
    const unsigned long long zero = dkey(0.0);
    cudaError_t e = cudaMemcpyAsync(c->gap_d, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    unsigned long long* gk = (unsigned long long*)c->gap_d;
    const RkGas g = rk_gas(c);
    if (c->D == 2) {
        if (c->mixed) rk_correct<2, float><<<c->Nc, RK_NT, 0, c->stream>>>(c->Nv, c->Nvp, (float*)f, c->xi_d, c->w_d,
                                                                           c->xi_f, c->w_f, Wtarget, g, iters, gk);
        else rk_correct<2, double><<<c->Nc, RK_NT, 0, c->stream>>>(c->Nv, c->Nvp, (double*)f, c->xi_d, c->w_d,
                                                                   c->xi_f, c->w_f, Wtarget, g, iters, gk);
    } else {
        if (c->mixed) rk_correct<3, float><<<c->Nc, RK_NT, 0, c->stream>>>(c->Nv, c->Nvp, (float*)f, c->xi_d, c->w_d,
                                                                           c->xi_f, c->w_f, Wtarget, g, iters, gk);
        else rk_correct<3, double><<<c->Nc, RK_NT, 0, c->stream>>>(c->Nv, c->Nvp, (double*)f, c->xi_d, c->w_d,
                                                                   c->xi_f, c->w_f, Wtarget, g, iters, gk);
    }
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t rk_launch_cons_to_prim(avs_ctx* c, const double* Wc, double* Wp)
{
    if (c->D == 2) rk_cons_to_prim<2><<<(c->Nc + 255) / 256, 256, 0, c->stream>>>(c->Nc, Wc, c->cfg.R, Wp);
    else rk_cons_to_prim<3><<<(c->Nc + 255) / 256, 256, 0, c->stream>>>(c->Nc, Wc, c->cfg.R, Wp);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace avs
