// One explicit UGKS step on the global velocity mesh (paper Sec. 2.3, with
// the explicit readings R1-R4), as two kernels.
//
// k_grad: the limited least-squares gradient L grad phi of every cell, array
//   and node (Sec. 2.3.3: least squares with weights 1/|d|^2, Venkatakrishnan
//   limiter), computed once and stored next to f.  Elementwise stencil over
//   the face neighbours.
//
// k_step: one thread block per physical cell, three passes over the nodes
// (thread t owns nodes k = t, t + NT, ...):
//   A  foot values phi_C + (L grad phi)_C . (x_f - xi h - x_C) of every face
//      from the upwind cell, summed into raw velocity moments per face
//      (interface W of Eq. w_interface, heat flux, flux moments).
//   -  interface Shakhov state per face: tau (Eq. 3), q_ij (R4), blend weights
//      tau/(tau+h), h/(tau+h) (Eq. equ28); incoming Maxwellians of boundaries.
//   B  interface equilibria: their discrete flux moments; the interface
//      distribution phi_ij = wa phi_bar + wb g_ij (foot values recomputed)
//      and the per-node net flux sum_j A (xi . n) phi_ij, parked in the
//      f^{n+1} slot of the node; raw moments of the cell's own f^n (lagged
//      heat flux, R3).  Wall density from zero net mass flux (R8).
//   -  W~ = W - dt/|V| sum_j A F_ij (R2) and the cell's Shakhov state.
//   C  collision update (diagonal of Eq. SGS_phi, R1), overwriting the slot.
//
// Faces shared by two cells are evaluated by both blocks from the same inputs
// with the same node-to-thread map and reduction order, so both copies of a
// face flux agree and W telescopes.  f^n, its gradient and W^n are read-only
// during the step, so blocks never wait on each other.  Sums: per-thread and
// warp sums in the element type, FP64 across warps and in every per-cell /
// per-face formula.
#include <algorithm>

#include "avs_dev.cuh"
#include "avs_internal.h"

namespace avs {

// ------------------------------------------------------------------ k_grad
// G[i][a][d][k] = L * (grad phi)_d of array a of cell i at node k.  Each
// thread handles VG consecutive nodes (rows are padded to 32 nodes, so the
// vector stays inside the row) to keep more loads in flight.
template <int D, typename T, int VG>
__global__ void __launch_bounds__(256) k_grad(int Nv, int Nvp, int limiter, const T* __restrict__ f,
                                              T* __restrict__ G, CellGeo<T> geo)
{
    constexpr int NA = NArr<D>::v;
    const int i = blockIdx.x;
    const int k0 = (blockIdx.y * blockDim.x + threadIdx.x) * VG;
    if (k0 >= Nv) return;
    const size_t cstride = (size_t)NA * Nvp;
    const int ns = geo.ns[i];
    int nb[AVS_MAXS];
    T cg[AVS_MAXS][D], rr[AVS_MAXS][D];
#pragma unroll
    for (int s = 0; s < AVS_MAXS; ++s) {
        nb[s] = s < ns ? geo.nbr[i * AVS_MAXS + s] : -1;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            cg[s][d] = s < ns ? geo.cg[(size_t)(i * AVS_MAXS + s) * D + d] : T(0);
            rr[s][d] = s < ns ? geo.r[(size_t)(i * AVS_MAXS + s) * D + d] : T(0);
        }
    }
    const T e2 = geo.eps2[i];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const T* fa = f + (size_t)a * Nvp + k0;
        T phi[VG], nv[AVS_MAXS][VG];
#pragma unroll
        for (int v = 0; v < VG; ++v) phi[v] = fa[(size_t)i * cstride + v];
#pragma unroll
        for (int s = 0; s < AVS_MAXS; ++s)
#pragma unroll
            for (int v = 0; v < VG; ++v) nv[s][v] = nb[s] >= 0 ? fa[(size_t)nb[s] * cstride + v] : phi[v];
        T* o = G + ((size_t)i * NA + a) * D * Nvp + k0;
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            T g[D];
#pragma unroll
            for (int d = 0; d < D; ++d) g[d] = T(0);
            T L = T(1);
            if (limiter != 0) {
                T dmax = T(0), dmin = T(0);
#pragma unroll
                for (int s = 0; s < AVS_MAXS; ++s) {
                    if (nb[s] < 0) continue;
                    const T dd = nv[s][v] - phi[v];
#pragma unroll
                    for (int d = 0; d < D; ++d) g[d] += cg[s][d] * dd;
                    dmax = dd > dmax ? dd : dmax;
                    dmin = dd < dmin ? dd : dmin;
                }
                if (limiter == 1) {
                    T p = T(0), n = T(0);
#pragma unroll
                    for (int s = 0; s < AVS_MAXS; ++s) {
                        if (s >= ns) break;
                        T d2 = g[0] * rr[s][0];
#pragma unroll
                        for (int d = 1; d < D; ++d) d2 += g[d] * rr[s][d];
                        p = d2 > p ? d2 : p;
                        n = d2 < n ? d2 : n;
                    }
                    if (p > T(0)) { const T t = venkat(dmax, p, e2); L = t < L ? t : L; }
                    if (n < T(0)) { const T t = venkat(dmin, n, e2); L = t < L ? t : L; }
                }
            }
            if (k0 + v < Nvp) {
#pragma unroll
                for (int d = 0; d < D; ++d) o[(size_t)d * Nvp + v] = L * g[d];
            }
        }
    }
}

// ------------------------------------------------------------------ k_step
template <int D, typename T>
struct StepP {
    int Nc, Nv, Nvp;
    size_t cstride;          // elements per cell in f: NA * Nvp
    T h;
    double dt, hd;
    double R, Pr, omega, mu_ref, T_ref;
    const T* __restrict__ fin;
    const T* __restrict__ G;   // [cell][array][dim][Nvp], null for first order
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
    const unsigned char* __restrict__ nslot;
    const double* __restrict__ vol;
    int* err;
};

template <typename T>
struct SlotSt {
    int kind, L, R;          // kind: 0 interior, 1 wall, 2 far field
    T sgn;                   // +1: the cell is L (An points out of it), -1: it is R
    T An[3], rL[3], rR[3];
    double And[3];
    double V[3];             // reference velocity of the moment sums
    T Vt[3];                 // the same in the element type
    EqPar<T> eq;             // interface equilibrium / incoming Maxwellian
    T wa, wb;
    double wad, wbd;
    double AF[5];            // area-weighted interface flux
};

template <typename A>
__device__ __forceinline__ A tau_vhs(A rho, A RT, A R, A mu_ref, A T_ref, A omega)
{
    const A T = RT / R;
    return mu_ref * powa(T / T_ref, omega) / (rho * RT);
}

// foot value of array a at node k from upwind cell C, offset rF of the face
template <int D, int NA, typename T>
__device__ __forceinline__ T foot(const StepP<D, T>& P, int C, int a, int k, const T* rF, const T* x, T h)
{
    T v = P.fin[(size_t)C * P.cstride + (size_t)a * P.Nvp + k];
    if (P.G) {
        const T* g = P.G + ((size_t)C * NA + a) * D * P.Nvp + k;
#pragma unroll
        for (int d = 0; d < D; ++d) v += g[(size_t)d * P.Nvp] * (rF[d] - x[d] * h);
    }
    return v;
}

template <int D> struct FaceGroup { static constexpr int v = (D == 2) ? 4 : 3; };

// nodes per thread per iteration: 16-byte vector loads along the node index
template <typename T> struct VW { static constexpr int v = 16 / sizeof(T); };

template <typename T, int V>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T* o)
{
    if constexpr (sizeof(T) == 4 && V == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    } else if constexpr (sizeof(T) == 8 && V == 2) {
        const double2 q = *reinterpret_cast<const double2*>(p);
        o[0] = q.x; o[1] = q.y;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) o[v] = p[v];
    }
}

template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const T* o)
{
    if constexpr (sizeof(T) == 4 && V == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(T) == 8 && V == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = o[v];
    }
}

// Foot values of both arrays at the V nodes k0.. from the upwind cells C[v]
// (vector loads when all V nodes share the upwind cell).
template <int D, int NA, int V, typename T>
__device__ __forceinline__ void foot_v(const StepP<D, T>& P, const int* C, int L, const T* rL, const T* rR, int k0,
                                       const T (*x)[D], T h, T (*out)[NA])
{
    bool uni = true;
#pragma unroll
    for (int v = 1; v < V; ++v) uni = uni && (C[v] == C[0]);
    T fv[NA][V], gv[NA][D][V];
    if (uni) {
        const size_t base = (size_t)C[0] * P.cstride + k0;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            ldv<T, V>(P.fin + base + (size_t)a * P.Nvp, fv[a]);
            if (P.G) {
                const T* g = P.G + ((size_t)C[0] * NA + a) * D * P.Nvp + k0;
#pragma unroll
                for (int d = 0; d < D; ++d) ldv<T, V>(g + (size_t)d * P.Nvp, gv[a][d]);
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                fv[a][v] = P.fin[(size_t)C[v] * P.cstride + (size_t)a * P.Nvp + k0 + v];
                if (P.G) {
                    const T* g = P.G + ((size_t)C[v] * NA + a) * D * P.Nvp + k0 + v;
#pragma unroll
                    for (int d = 0; d < D; ++d) gv[a][d][v] = g[(size_t)d * P.Nvp];
                }
            }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const T* r = C[v] == L ? rL : rR;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            T val = fv[a][v];
            if (P.G) {
#pragma unroll
                for (int d = 0; d < D; ++d) val += gv[a][d][v] * (r[d] - x[v][d] * h);
            }
            out[v][a] = val;
        }
    }
}

template <int D, int V, typename T>
__device__ __forceinline__ void load_nodes(const StepP<D, T>& P, int k0, T (*x)[D], T* w)
{
    T xx[V * D];
    if constexpr ((V * D * sizeof(T)) % 16 == 0) {
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int j = 0; j < V * D / PER; ++j) ldv<T, PER>(P.xi + (size_t)k0 * D + j * PER, xx + j * PER);
    } else {
#pragma unroll
        for (int j = 0; j < V * D; ++j) xx[j] = P.xi[(size_t)k0 * D + j];
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
        for (int d = 0; d < D; ++d) x[v][d] = xx[v * D + d];
    ldv<T, V>(P.w + k0, w);
}

template <int D, typename T, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4) ? 4 : 1) k_step(StepP<D, T> P)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    constexpr int FG = FaceGroup<D>::v;                  // faces per pass-A sweep
    constexpr int NB = AVS_MAXS * (NW + 1) + NM;         // values reduced after pass B
    constexpr int NR = (FG * NM > NB) ? FG * NM : NB;
    constexpr int V = VW<T>::v;
    __shared__ SlotSt<T> S[AVS_MAXS];
    __shared__ double sw[(NT / 32) * NR];
    __shared__ double red[NR];
    __shared__ double mom[AVS_MAXS][NM];
    __shared__ double Vc[3], qc[3];
    __shared__ EqPar<T> ceq;
    __shared__ T upd[4];
    __shared__ int wall_slots[AVS_MAXS], n_wall;

    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const T h = P.h;
    const int ns = P.nslot[i];
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        const int f = sl >> 1;
        SlotSt<T>& s = S[tid];
        s.L = P.faceL[f];
        s.R = P.faceR[f];
        s.sgn = (sl & 1) ? T(-1) : T(1);
        s.kind = s.R >= 0 ? 0 : (int)P.bc[(size_t)(-1 - s.R) * 6];
        for (int d = 0; d < 3; ++d) {
            s.An[d] = d < D ? P.An[(size_t)f * D + d] : T(0);
            s.And[d] = d < D ? P.An_d[(size_t)f * D + d] : 0.0;
            s.rL[d] = d < D ? P.rL[(size_t)f * D + d] : T(0);
            s.rR[d] = d < D ? P.rR[(size_t)f * D + d] : T(0);
            T v = T(0);
            if (d < D) {
                v = (T)P.Win[(size_t)s.L * NW + 1 + d] / (T)P.Win[(size_t)s.L * NW];
                if (s.R >= 0) v = T(0.5) * (v + (T)P.Win[(size_t)s.R * NW + 1 + d] / (T)P.Win[(size_t)s.R * NW]);
            }
            s.V[d] = (double)v;
            s.Vt[d] = v;
        }
    }
    if (tid == 0) {
        for (int d = 0; d < 3; ++d)
            Vc[d] = d < D ? (double)((T)P.Win[(size_t)i * NW + 1 + d] / (T)P.Win[(size_t)i * NW]) : 0.0;
        int nw = 0;
        for (int s = 0; s < ns; ++s) {
            const int R = P.faceR[P.slot[i * AVS_MAXS + s] >> 1];
            if (R < 0 && (int)P.bc[(size_t)(-1 - R) * 6] == AVS_BC_WALL) wall_slots[nw++] = s;
        }
        n_wall = nw;
    }
    __syncthreads();

    // ---------------- pass A: raw moments of the foot distribution, FG faces per sweep
    for (int s0 = 0; s0 < ns; s0 += FG) {
        const int s1 = min(ns, s0 + FG);
        T acc[FG * NM];
#pragma unroll
        for (int m = 0; m < FG * NM; ++m) acc[m] = T(0);
        for (int k0 = tid * V; k0 < P.Nv; k0 += NT * V) {
            T x[V][D], wv[V];
            load_nodes<D, V>(P, k0, x, wv);      // pad nodes carry w = 0 and contribute nothing
#pragma unroll
            for (int j = 0; j < FG; ++j) {
                const int s = s0 + j;
                if (s >= s1) break;
                const SlotSt<T>& Sl = S[s];
                T An[D];
#pragma unroll
                for (int d = 0; d < D; ++d) An[d] = Sl.An[d];
                const bool inter = Sl.kind == 0;
                T sn[V];
                int C[V];
                bool any = false;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    sn[v] = dot_rn<D>(x[v], An);
                    C[v] = (sn[v] >= T(0) || !inter) ? Sl.L : Sl.R;
                    any = any || inter || sn[v] >= T(0);
                }
                if (!any) continue;                 // all incoming at a boundary: pass B
                T fv[V][NA];
                foot_v<D, NA, V>(P, C, Sl.L, Sl.rL, Sl.rR, k0, x, h, fv);
                T* m = acc + j * NM;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if (inter) {
                        T xs[D];
#pragma unroll
                        for (int d = 0; d < D; ++d) xs[d] = x[v][d] - Sl.Vt[d];
                        raw_acc<D>(m, xs, wv[v] * fv[v][0], NA == 2 ? wv[v] * fv[v][NA - 1] : T(0));
                    } else if (sn[v] >= T(0)) {
                        const T t = wv[v] * sn[v];
                        T x2 = T(0);
#pragma unroll
                        for (int d = 0; d < D; ++d) x2 += x[v][d] * x[v][d];
                        m[0] += t * fv[v][0];
#pragma unroll
                        for (int d = 0; d < D; ++d) m[1 + d] += t * fv[v][0] * x[v][d];
                        m[D + 1] += t * T(0.5) * (x2 * fv[v][0] + (NA == 2 ? fv[v][NA - 1] : T(0)));
                    }
                }
            }
        }
        block_sum_t<FG * NM, NT>(acc, sw, red);
        for (int v = tid; v < (s1 - s0) * NM; v += NT) mom[s0 + v / NM][v % NM] = red[v];
        __syncthreads();
    }

    // ---------------- interface states
    if (tid < ns) {
        SlotSt<T>& s = S[tid];
        if (s.kind == 0) {
            double Wd[5], AFphi[5];
            moments_from_raw<D>(mom[tid], s.V, Wd, nullptr, s.And, AFphi);
            T rho, U[3], RT, qb[3];
            state_from_raw<D, T>(mom[tid], s.V, rho, U, RT, qb);
            if (!(rho > T(0)) || !(RT > T(0))) atomicOr(P.err, 1);
            const T tau = tau_vhs<T>(rho, RT, (T)P.R, (T)P.mu_ref, (T)P.T_ref, (T)P.omega);
            const T hh = (T)P.hd;
            T qf[3] = {T(0), T(0), T(0)};
            for (int d = 0; d < D; ++d) qf[d] = tau * qb[d] / (tau + hh * (T)P.Pr);
            s.eq = make_eq_a<D, T, T>(rho, U, RT, qf, (T)P.Pr);
            s.wad = (double)(tau / (tau + hh));
            s.wbd = (double)(hh / (tau + hh));
            for (int m = 0; m < NW; ++m) s.AF[m] = s.wad * AFphi[m];
        } else {
            const double* B = P.bc + (size_t)(-1 - s.R) * 6;
            const double Ub[3] = {B[2], B[3], B[4]};
            s.eq = make_eq<D, T>(s.kind == 1 ? 1.0 : B[1], Ub, P.R * B[5], nullptr, P.Pr);
            s.wad = 1.0;
            s.wbd = 0.0;
            for (int m = 0; m < NW; ++m) s.AF[m] = mom[tid][m];   // outgoing half
        }
        s.wa = (T)s.wad;
        s.wb = (T)s.wbd;
    }
    __syncthreads();

    // ---------------- pass B: face equilibria, interface distribution, net flux, cell moments
    const T* fi = P.fin + (size_t)i * P.cstride;
    T* fo = P.fout + (size_t)i * P.cstride;
    {
        T acc[NB];
#pragma unroll
        for (int m = 0; m < NB; ++m) acc[m] = T(0);
        T Vct[D];
#pragma unroll
        for (int d = 0; d < D; ++d) Vct[d] = (T)Vc[d];
        for (int k0 = tid * V; k0 < P.Nv; k0 += NT * V) {
            T x[V][D], wv[V], x2[V];
            load_nodes<D, V>(P, k0, x, wv);
            {
                T f0[V], f1[V];
                ldv<T, V>(fi + k0, f0);
                if (NA == 2) ldv<T, V>(fi + P.Nvp + k0, f1);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    T xs[D];
                    x2[v] = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        xs[d] = x[v][d] - Vct[d];
                        x2[v] += x[v][d] * x[v][d];
                    }
                    raw_acc<D>(acc + AVS_MAXS * (NW + 1), xs, wv[v] * f0[v], NA == 2 ? wv[v] * f1[v] : T(0));
                }
            }
            T Nn[NA][V];
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int v = 0; v < V; ++v) Nn[a][v] = T(0);
#pragma unroll
            for (int s = 0; s < AVS_MAXS; ++s) {
                if (s >= ns) break;
                const SlotSt<T>& Sl = S[s];
                T An[D];
#pragma unroll
                for (int d = 0; d < D; ++d) An[d] = Sl.An[d];
                T sn[V];
                int C[V];
                bool need_foot = false;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    sn[v] = dot_rn<D>(x[v], An);
                    C[v] = (sn[v] >= T(0) || Sl.kind != 0) ? Sl.L : Sl.R;
                    need_foot = need_foot || Sl.kind == 0 || sn[v] >= T(0);
                }
                T fv[V][NA];
                if (need_foot) foot_v<D, NA, V>(P, C, Sl.L, Sl.rL, Sl.rR, k0, x, h, fv);
                T* m = acc + s * (NW + 1);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const T ss = Sl.sgn * sn[v];
                    if (Sl.kind != 0 && sn[v] >= T(0)) {     // outgoing at a boundary: the foot value
#pragma unroll
                        for (int a = 0; a < NA; ++a) Nn[a][v] += ss * fv[v][a];
                        continue;
                    }
                    T gG, gH;
                    eq_eval<D>(Sl.eq, x[v], gG, gH);
                    const T t = wv[v] * sn[v];
                    m[0] += t * gG;
#pragma unroll
                    for (int d = 0; d < D; ++d) m[1 + d] += t * gG * x[v][d];
                    m[D + 1] += t * T(0.5) * (x2[v] * gG + gH);
                    if (Sl.kind == 0) {
                        Nn[0][v] += ss * (Sl.wa * fv[v][0] + Sl.wb * gG);
                        if (NA == 2) Nn[NA - 1][v] += ss * (Sl.wa * fv[v][NA - 1] + Sl.wb * gH);
                    } else if (Sl.kind == 2) {
                        Nn[0][v] += ss * gG;
                        if (NA == 2) Nn[NA - 1][v] += ss * gH;
                    } else {
                        m[NW] += wv[v] * (-sn[v]) * gG;          // wall: incoming part added in pass C
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) stv<T, V>(fo + (size_t)a * P.Nvp + k0, Nn[a]);   // parked until pass C
        }
        block_sum_t<NB, NT>(acc, sw, red);
    }

    // ---------------- final interface fluxes, wall densities, lagged heat flux
    if (tid < ns) {
        SlotSt<T>& s = S[tid];
        const double* g = red + tid * (NW + 1);
        if (s.kind == 0) {
            for (int m = 0; m < NW; ++m) s.AF[m] += s.wbd * g[m];
        } else if (s.kind == 1) {
            const double Sin = g[NW];
            const double rw = Sin > 0.0 ? s.AF[0] / Sin : 0.0;
            for (int m = 0; m < NW; ++m) s.AF[m] += rw * g[m];
            const double* B = P.bc + (size_t)(-1 - s.R) * 6;
            const double Ub[3] = {B[2], B[3], B[4]};
            s.eq = make_eq<D, T>(rw, Ub, P.R * B[5], nullptr, P.Pr);
        } else {
            for (int m = 0; m < NW; ++m) s.AF[m] += g[m];
        }
    }
    if (tid == 32 % NT) {
        T rn, Un[3], RTn, qn[3];
        state_from_raw<D, T>(red + AVS_MAXS * (NW + 1), Vc, rn, Un, RTn, qn);
        for (int d = 0; d < 3; ++d) qc[d] = d < D ? (double)qn[d] : 0.0;
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
        double rhod, Ud[3], RTd;
        prim<D>(Wt, rhod, Ud, RTd);
        if (!(rhod > 0.0) || !(RTd > 0.0)) atomicOr(P.err, 1);
        const T rho = (T)rhod, RT = (T)RTd;
        T U[3], q[3];
        for (int d = 0; d < 3; ++d) {
            U[d] = (T)Ud[d];
            q[d] = (T)qc[d];
        }
        const T tau = tau_vhs<T>(rho, RT, (T)P.R, (T)P.mu_ref, (T)P.T_ref, (T)P.omega);
        ceq = make_eq_a<D, T, T>(rho, U, RT, q, (T)P.Pr);
        const T idt = (T)(1.0 / P.dt), itau = T(1) / tau;
        upd[0] = idt;
        upd[1] = itau;
        upd[2] = (T)(1.0 / P.vol[i]);
        upd[3] = T(1) / (idt + itau);
    }
    __syncthreads();

    // ---------------- pass C: collision update (pad nodes are written as zero)
    const int nw = n_wall;
    for (int k0 = tid * V; k0 < P.Nv; k0 += NT * V) {
        T x[V][D], wv[V];
        load_nodes<D, V>(P, k0, x, wv);
        T Nn[NA][V], fv[NA][V], out[NA][V];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            ldv<T, V>(fo + (size_t)a * P.Nvp + k0, Nn[a]);
            ldv<T, V>(fi + (size_t)a * P.Nvp + k0, fv[a]);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            for (int j = 0; j < nw; ++j) {
                const SlotSt<T>& Sl = S[wall_slots[j]];
                T An[D];
#pragma unroll
                for (int d = 0; d < D; ++d) An[d] = Sl.An[d];
                const T sn = dot_rn<D>(x[v], An);
                if (sn >= T(0)) continue;
                T gG, gH;
                eq_eval<D>(Sl.eq, x[v], gG, gH);
                const T ss = Sl.sgn * sn;
                Nn[0][v] += ss * gG;
                if (NA == 2) Nn[NA - 1][v] += ss * gH;
            }
            T gG, gH;
            eq_eval<D>(ceq, x[v], gG, gH);
            const bool real = k0 + v < P.Nv;
            out[0][v] = real ? (fv[0][v] * upd[0] + gG * upd[1] - Nn[0][v] * upd[2]) * upd[3] : T(0);
            if (NA == 2)
                out[NA - 1][v] = real ? (fv[NA - 1][v] * upd[0] + gH * upd[1] - Nn[NA - 1][v] * upd[2]) * upd[3] : T(0);
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) stv<T, V>(fo + (size_t)a * P.Nvp + k0, out[a]);
    }
}

template <int D, typename T>
static cudaError_t launch_step_t(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout,
                                 double dt)
{
    const bool f32 = sizeof(T) == 4;
    const int NA = NArr<D>::v;
    const bool grad = c->cfg.limiter != 0;
    if (grad) {
        // sized for the f capacity so that adaptation does not reallocate it
        const size_t need = (size_t)c->Nc * NA * D * std::max(c->fcap, c->Nvp) * sizeof(T);
        if (c->grad_bytes < need) {
            if (c->grad) cudaFree(c->grad);
            c->grad = nullptr;
            c->grad_bytes = 0;
            cudaError_t e = cudaMalloc(&c->grad, need);
            if (e != cudaSuccess) return e;
            c->grad_bytes = need;
        }
        CellGeo<T> geo;
        geo.nbr = c->nbr;
        geo.cg = f32 ? (const T*)c->cg_f : (const T*)c->cg_d;
        geo.r = f32 ? (const T*)c->r_f : (const T*)c->r_d;
        geo.eps2 = f32 ? (const T*)c->eps2_f : (const T*)c->eps2_d;
        geo.ns = c->nslot;
        constexpr int VG = 4;
        dim3 g(c->Nc, (c->Nv + 256 * VG - 1) / (256 * VG));
        k_grad<D, T, VG><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (const T*)fin, (T*)c->grad, geo);
        c->launches += 1;
    }
    StepP<D, T> P;
    P.Nc = c->Nc;
    P.Nv = c->Nv;
    P.Nvp = c->Nvp;
    P.cstride = (size_t)NA * c->Nvp;
    P.dt = dt;
    P.hd = 0.5 * dt;
    P.h = (T)P.hd;
    P.R = c->cfg.R;
    P.Pr = c->cfg.Pr;
    P.omega = c->cfg.omega;
    P.mu_ref = c->mu_ref;
    P.T_ref = c->cfg.T_ref;
    P.fin = (const T*)fin;
    P.G = grad ? (const T*)c->grad : nullptr;
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
    P.nslot = c->nslot;
    P.vol = c->vol;
    P.err = c->dev_err;
    constexpr int NT = sizeof(T) == 4 ? 128 : 256;
    k_step<D, T, NT><<<c->Nc, NT, 0, c->stream>>>(P);
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
