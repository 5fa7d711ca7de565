// One explicit UGKS step on the global velocity mesh (paper Sec. 2.3, with
// the explicit readings R1-R4): one thread block per physical cell.
//
//   pass 1a  for every face of the cell: foot values phi_C + L grad.(x_f - xi h - x_C)
//            from the upwind cell (Sec. 2.3.3), summed into raw velocity
//            moments (interface W of Eq. w_interface, heat flux, flux moments)
//   pass 1b  raw moments of the cell's own f^n (lagged heat flux, R3)
//   state    interface Shakhov state per face: tau (Eq. 3), q_ij (R4), blend
//            weights tau/(tau+h), h/(tau+h) (Eq. equ28); wall density from
//            zero net mass flux (R8)
//   pass 1c  discrete flux moments of the interface equilibrium
//   update   W~ = W - dt/|V| sum_j A F_ij (R2), cell Shakhov state
//   pass 2   phi_ij per node and face, net flux, collision update (Eq. SGS_phi
//            diagonal, R1), written to the second f buffer.
//
// Faces shared by two cells are evaluated by both blocks with identical
// arithmetic (same inputs, same node-to-thread map, same reduction order), so
// the two flux copies agree bit for bit and W telescopes.  f^n and W^n are
// read-only during the step (double buffers), so blocks never wait on each
// other.
#include "avs_dev.cuh"
#include "avs_internal.h"

namespace avs {

template <int D, typename T>
struct StepP {
    int Nv, Nvp, limiter;
    size_t cstride;
    T h;
    double dt, hd;
    double R, Pr, omega, mu_ref, T_ref;
    const T* __restrict__ fin;
    T* __restrict__ fout;
    const double* __restrict__ Win;
    double* __restrict__ Wout;
    const T* __restrict__ xi;
    const T* __restrict__ w;
    const int* __restrict__ faceL;
    const int* __restrict__ faceR;
    const T* __restrict__ An;
    const double* __restrict__ An_d;
    const T* __restrict__ rL;
    const T* __restrict__ rR;
    const double* __restrict__ bc;
    const int* __restrict__ slot;
    const double* __restrict__ vol;
    CellGeo<T> geo;
    int* err;
};

template <typename T>
struct SlotSt {
    int kind, f, L, R;       // kind: 0 interior, 1 wall, 2 far field
    T sgn;                   // +1: the cell is L (An points out of it), -1: it is R
    T An[3], rL[3], rR[3];
    double And[3];
    double V[3];             // reference velocity of the moment sums
    EqPar<T> eq;             // interface equilibrium / incoming Maxwellian
    T wa, wb;
    double wad, wbd;
    double mom[13];          // raw moments of the foot distribution / outgoing flux
    double AFphi[5];
    double AFg[6];
    double AF[5];            // area-weighted interface flux
};

__device__ __forceinline__ double tau_vhs(double rho, double RT, double R, double mu_ref, double T_ref,
                                          double omega)
{
    const double T = RT / R;
    return mu_ref * pow(T / T_ref, omega) / (rho * RT);
}

template <int D, typename T, int NT>
__global__ void __launch_bounds__(NT) k_step(StepP<D, T> P)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    // FP32 partial sums are flushed into FP64 every CH nodes per thread.
    constexpr int CH = (sizeof(T) == 4) ? 8 : (1 << 20);
    __shared__ SlotSt<T> S[AVS_MAXS];
    __shared__ double sred[(NT / 32) * 14];
    __shared__ double cmom[NM];
    __shared__ double Vc[3], qc[3];
    __shared__ EqPar<T> ceq;
    __shared__ T upd[4];

    const int i = blockIdx.x, tid = threadIdx.x;
    const int ns = P.geo.ns[i];
    const T h = P.h;

    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        SlotSt<T>& s = S[tid];
        s.f = sl >> 1;
        s.L = P.faceL[s.f];
        s.R = P.faceR[s.f];
        s.sgn = (sl & 1) ? T(-1) : T(1);
        s.kind = s.R >= 0 ? 0 : (int)P.bc[(size_t)(-1 - s.R) * 6];
        for (int d = 0; d < 3; ++d) {
            s.An[d] = d < D ? P.An[(size_t)s.f * D + d] : T(0);
            s.And[d] = d < D ? P.An_d[(size_t)s.f * D + d] : 0.0;
            s.rL[d] = d < D ? P.rL[(size_t)s.f * D + d] : T(0);
            s.rR[d] = d < D ? P.rR[(size_t)s.f * D + d] : T(0);
            double v = 0.0;
            if (d < D) {
                v = P.Win[(size_t)s.L * NW + 1 + d] / P.Win[(size_t)s.L * NW];
                if (s.R >= 0) v = 0.5 * (v + P.Win[(size_t)s.R * NW + 1 + d] / P.Win[(size_t)s.R * NW]);
            }
            s.V[d] = (double)(T)v;
        }
    }
    if (tid == 0) {
        for (int d = 0; d < 3; ++d)
            Vc[d] = d < D ? (double)(T)(P.Win[(size_t)i * NW + 1 + d] / P.Win[(size_t)i * NW]) : 0.0;
    }
    __syncthreads();

    // ---------------- pass 1a: raw moments of the foot distribution per face
    for (int s = 0; s < ns; ++s) {
        const int L = S[s].L, R = S[s].R;
        const bool inter = S[s].kind == 0;
        T An[D], rLs[D], rRs[D], Vt[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            An[d] = S[s].An[d];
            rLs[d] = S[s].rL[d];
            rRs[d] = S[s].rR[d];
            Vt[d] = (T)S[s].V[d];
        }
        double acc[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = 0.0;
        for (int k0 = tid; k0 < P.Nv; k0 += NT * CH) {
            T part[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) part[m] = T(0);
            for (int c = 0, k = k0; c < CH && k < P.Nv; ++c, k += NT) {
                T x[D];
#pragma unroll
                for (int d = 0; d < D; ++d) x[d] = P.xi[(size_t)k * D + d];
                const T sn = dot_rn<D>(x, An);
                int C;
                const T* rF;
                if (sn >= T(0)) { C = L; rF = rLs; }
                else if (inter) { C = R; rF = rRs; }
                else continue;
                T gr[D], Lm;
                const T phiG = grad_lim<D>(P.geo, P.limiter, P.fin + k, P.cstride, C, gr, Lm);
                const T fG = foot_value<D>(phiG, gr, Lm, rF, x, h);
                T fH = T(0);
                if (NA == 2) {
                    const T phiH = grad_lim<D>(P.geo, P.limiter, P.fin + P.Nvp + k, P.cstride, C, gr, Lm);
                    fH = foot_value<D>(phiH, gr, Lm, rF, x, h);
                }
                const T wk = P.w[k];
                if (inter) {
                    T xs[D];
#pragma unroll
                    for (int d = 0; d < D; ++d) xs[d] = x[d] - Vt[d];
                    raw_acc<D>(part, xs, wk * fG, wk * fH);
                } else {
                    const T t = wk * sn;
                    T x2 = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) x2 += x[d] * x[d];
                    part[0] += t * fG;
#pragma unroll
                    for (int d = 0; d < D; ++d) part[1 + d] += t * fG * x[d];
                    part[D + 1] += t * T(0.5) * (x2 * fG + fH);
                }
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) acc[m] += (double)part[m];
        }
        block_sum<NM, NT>(acc, sred, S[s].mom);
    }

    // ---------------- pass 1b: raw moments of the cell's own f^n
    {
        double acc[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = 0.0;
        T Vt[D];
#pragma unroll
        for (int d = 0; d < D; ++d) Vt[d] = (T)Vc[d];
        const T* fi = P.fin + (size_t)i * P.cstride;
        for (int k0 = tid; k0 < P.Nv; k0 += NT * CH) {
            T part[NM];
#pragma unroll
            for (int m = 0; m < NM; ++m) part[m] = T(0);
            for (int c = 0, k = k0; c < CH && k < P.Nv; ++c, k += NT) {
                T xs[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xs[d] = P.xi[(size_t)k * D + d] - Vt[d];
                const T wk = P.w[k];
                raw_acc<D>(part, xs, wk * fi[k], NA == 2 ? wk * fi[P.Nvp + k] : T(0));
            }
#pragma unroll
            for (int m = 0; m < NM; ++m) acc[m] += (double)part[m];
        }
        block_sum<NM, NT>(acc, sred, cmom);
    }

    // ---------------- interface states and the cell's lagged heat flux
    if (tid < ns) {
        SlotSt<T>& s = S[tid];
        if (s.kind == 0) {
            double W[5], qb[3], rho, U[3], RT;
            moments_from_raw<D>(s.mom, s.V, W, qb, s.And, s.AFphi);
            prim<D>(W, rho, U, RT);
            if (!(rho > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
            const double tau = tau_vhs(rho, RT, P.R, P.mu_ref, P.T_ref, P.omega);
            double qf[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) qf[d] = tau * qb[d] / (tau + P.hd * P.Pr);
            s.eq = make_eq<D, T>(rho, U, RT, qf, P.Pr);
            s.wad = tau / (tau + P.hd);
            s.wbd = P.hd / (tau + P.hd);
        } else {
            for (int m = 0; m < NW; ++m) s.AFphi[m] = s.mom[m];
            const double* B = P.bc + (size_t)(-1 - s.R) * 6;
            const double Ub[3] = {B[2], B[3], B[4]};
            s.eq = make_eq<D, T>(s.kind == 1 ? 1.0 : B[1], Ub, P.R * B[5], nullptr, P.Pr);
            s.wad = 1.0;
            s.wbd = 0.0;
        }
        s.wa = (T)s.wad;
        s.wb = (T)s.wbd;
    }
    if (tid == 32) {
        double Wn[5], qn[3];
        moments_from_raw<D>(cmom, Vc, Wn, qn, nullptr, nullptr);
        for (int d = 0; d < 3; ++d) qc[d] = d < D ? qn[d] : 0.0;
    }
    __syncthreads();

    // ---------------- pass 1c: discrete flux moments of the face equilibria
    for (int s = 0; s < ns; ++s) {
        const int kind = S[s].kind;
        const EqPar<T> eq = S[s].eq;
        T An[D];
#pragma unroll
        for (int d = 0; d < D; ++d) An[d] = S[s].An[d];
        double acc[NW + 1];
#pragma unroll
        for (int m = 0; m <= NW; ++m) acc[m] = 0.0;
        for (int k0 = tid; k0 < P.Nv; k0 += NT * CH) {
            T part[NW + 1];
#pragma unroll
            for (int m = 0; m <= NW; ++m) part[m] = T(0);
            for (int c = 0, k = k0; c < CH && k < P.Nv; ++c, k += NT) {
                T x[D];
#pragma unroll
                for (int d = 0; d < D; ++d) x[d] = P.xi[(size_t)k * D + d];
                const T sn = dot_rn<D>(x, An);
                if (kind != 0 && sn >= T(0)) continue;
                T gG, gH;
                eq_eval<D>(eq, x, gG, gH);
                const T wk = P.w[k];
                const T t = wk * sn;
                T x2 = T(0);
#pragma unroll
                for (int d = 0; d < D; ++d) x2 += x[d] * x[d];
                part[0] += t * gG;
#pragma unroll
                for (int d = 0; d < D; ++d) part[1 + d] += t * gG * x[d];
                part[D + 1] += t * T(0.5) * (x2 * gG + gH);
                if (kind == 1) part[NW] += wk * (-sn) * gG;
            }
#pragma unroll
            for (int m = 0; m <= NW; ++m) acc[m] += (double)part[m];
        }
        block_sum<NW + 1, NT>(acc, sred, S[s].AFg);
    }

    // ---------------- final interface fluxes
    if (tid < ns) {
        SlotSt<T>& s = S[tid];
        if (s.kind == 0) {
            for (int m = 0; m < NW; ++m) s.AF[m] = s.wad * s.AFphi[m] + s.wbd * s.AFg[m];
        } else if (s.kind == 1) {
            const double Sin = s.AFg[NW];
            const double rw = Sin > 0.0 ? s.AFphi[0] / Sin : 0.0;
            for (int m = 0; m < NW; ++m) s.AF[m] = s.AFphi[m] + rw * s.AFg[m];
            const double* B = P.bc + (size_t)(-1 - s.R) * 6;
            const double Ub[3] = {B[2], B[3], B[4]};
            s.eq = make_eq<D, T>(rw, Ub, P.R * B[5], nullptr, P.Pr);
        } else {
            for (int m = 0; m < NW; ++m) s.AF[m] = s.AFphi[m] + s.AFg[m];
        }
    }
    __syncthreads();

    // ---------------- macroscopic predictor and the cell equilibrium
    if (tid == 0) {
        const double* Wi = P.Win + (size_t)i * NW;
        double Wt[5];
        const double dtv = P.dt / P.vol[i];
        for (int c = 0; c < NW; ++c) {
            double sum = 0.0;
            for (int s = 0; s < ns; ++s) sum += (double)S[s].sgn * S[s].AF[c];
            Wt[c] = Wi[c] - dtv * sum;
            P.Wout[(size_t)i * NW + c] = Wt[c];
        }
        double rho, U[3], RT;
        prim<D>(Wt, rho, U, RT);
        if (!(rho > 0.0) || !(RT > 0.0)) atomicOr(P.err, 1);
        const double tau = tau_vhs(rho, RT, P.R, P.mu_ref, P.T_ref, P.omega);
        ceq = make_eq<D, T>(rho, U, RT, qc, P.Pr);
        upd[0] = (T)(1.0 / P.dt);
        upd[1] = (T)(1.0 / tau);
        upd[2] = (T)(1.0 / P.vol[i]);
        upd[3] = (T)(1.0 / (1.0 / P.dt + 1.0 / tau));
    }
    __syncthreads();

    // ---------------- pass 2: interface distribution, net flux, collision update
    T* fo = P.fout + (size_t)i * P.cstride;
    for (int k = tid; k < P.Nv; k += NT) {
        T x[D];
#pragma unroll
        for (int d = 0; d < D; ++d) x[d] = P.xi[(size_t)k * D + d];
        T grG[D], LG, grH[D], LH = T(1);
        const T phiG = grad_lim<D>(P.geo, P.limiter, P.fin + k, P.cstride, i, grG, LG);
        T phiH = T(0);
        if (NA == 2) phiH = grad_lim<D>(P.geo, P.limiter, P.fin + P.Nvp + k, P.cstride, i, grH, LH);
        T NG = T(0), NH = T(0);
        for (int s = 0; s < ns; ++s) {
            const SlotSt<T>& Sl = S[s];
            T An[D];
#pragma unroll
            for (int d = 0; d < D; ++d) An[d] = Sl.An[d];
            const T sn = dot_rn<D>(x, An);
            T pG, pH = T(0);
            if (Sl.kind == 0) {
                const int C = sn >= T(0) ? Sl.L : Sl.R;
                const T* rF = sn >= T(0) ? Sl.rL : Sl.rR;
                T fG, fH = T(0);
                if (C == i) {
                    fG = foot_value<D>(phiG, grG, LG, rF, x, h);
                    if (NA == 2) fH = foot_value<D>(phiH, grH, LH, rF, x, h);
                } else {
                    T gr[D], Lm;
                    const T pg = grad_lim<D>(P.geo, P.limiter, P.fin + k, P.cstride, C, gr, Lm);
                    fG = foot_value<D>(pg, gr, Lm, rF, x, h);
                    if (NA == 2) {
                        const T ph = grad_lim<D>(P.geo, P.limiter, P.fin + P.Nvp + k, P.cstride, C, gr, Lm);
                        fH = foot_value<D>(ph, gr, Lm, rF, x, h);
                    }
                }
                T gG, gH;
                eq_eval<D>(Sl.eq, x, gG, gH);
                pG = Sl.wa * fG + Sl.wb * gG;
                pH = Sl.wa * fH + Sl.wb * gH;
            } else if (sn >= T(0)) {
                pG = foot_value<D>(phiG, grG, LG, Sl.rL, x, h);
                if (NA == 2) pH = foot_value<D>(phiH, grH, LH, Sl.rL, x, h);
            } else {
                eq_eval<D>(Sl.eq, x, pG, pH);
            }
            const T ss = Sl.sgn * sn;
            NG += ss * pG;
            NH += ss * pH;
        }
        T gG, gH;
        eq_eval<D>(ceq, x, gG, gH);
        fo[k] = (phiG * upd[0] + gG * upd[1] - NG * upd[2]) * upd[3];
        if (NA == 2) fo[P.Nvp + k] = (phiH * upd[0] + gH * upd[1] - NH * upd[2]) * upd[3];
    }
}

template <int D, typename T>
static cudaError_t launch_step_t(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout,
                                 double dt)
{
    StepP<D, T> P;
    const bool f32 = sizeof(T) == 4;
    P.Nv = c->Nv;
    P.Nvp = c->Nvp;
    P.limiter = c->cfg.limiter;
    P.cstride = (size_t)c->NA * c->Nvp;
    P.dt = dt;
    P.hd = 0.5 * dt;
    P.h = (T)P.hd;
    P.R = c->cfg.R;
    P.Pr = c->cfg.Pr;
    P.omega = c->cfg.omega;
    P.mu_ref = c->mu_ref;
    P.T_ref = c->cfg.T_ref;
    P.fin = (const T*)fin;
    P.fout = (T*)fout;
    P.Win = Win;
    P.Wout = Wout;
    P.xi = f32 ? (const T*)c->xi_f : (const T*)c->xi_d;
    P.w = f32 ? (const T*)c->w_f : (const T*)c->w_d;
    P.faceL = c->faceL;
    P.faceR = c->faceR;
    P.An = f32 ? (const T*)c->An_f : (const T*)c->An_d;
    P.An_d = c->An_d;
    P.rL = f32 ? (const T*)c->rL_f : (const T*)c->rL_d;
    P.rR = f32 ? (const T*)c->rR_f : (const T*)c->rR_d;
    P.bc = c->bc;
    P.slot = c->slot;
    P.vol = c->vol;
    P.geo.nbr = c->nbr;
    P.geo.cg = f32 ? (const T*)c->cg_f : (const T*)c->cg_d;
    P.geo.r = f32 ? (const T*)c->r_f : (const T*)c->r_d;
    P.geo.eps2 = f32 ? (const T*)c->eps2_f : (const T*)c->eps2_d;
    P.geo.ns = c->nslot;
    P.err = c->dev_err;
    k_step<D, T, AVS_NT><<<c->Nc, AVS_NT, 0, c->stream>>>(P);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_step(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt)
{
    if (c->D == 2)
        return c->mixed ? launch_step_t<2, float>(c, fin, fout, Win, Wout, dt)
                        : launch_step_t<2, double>(c, fin, fout, Win, Wout, dt);
    return c->mixed ? launch_step_t<3, float>(c, fin, fout, Win, Wout, dt)
                    : launch_step_t<3, double>(c, fin, fout, Win, Wout, dt);
}

}  // namespace avs
