// Velocity-mesh kernels: node geometry, time-step bound, initial field,
// moments, adaptive criterion, split/merge marks with prefix-scan compaction,
// consanguinity remap and conservation correction (paper Sec. 3).
//
// The criterion, the marks and the new tree are computed with the same
// operation order as a plain sequential code, without fused multiply-adds,
// so that for the same f and W the adapted topology is bit-identical.
#include <string.h>

#include "avs_dev.cuh"
#include "avs_internal.h"

namespace avs {

int round_up(int n, int m) { return (n + m - 1) / m * m; }

// ------------------------------------------------------------------ geometry
// Mid-point quadrature on the tree (Sec. 3): node = element centre,
// weight = element area/volume; xi = vlo + hb (b + (2o+1)/2^(l+1)).
// The node's refinement cap: the largest level of the zones holding its
// centre (r_in^2 <= |xi - c|^2 < r_out^2, FP64 without contraction), else the
// outside level; max_refine when no zones are set (Sec. 3.5).
__device__ int zone_cap(const ZoneSet& Z, int D, const double* x)
{
    if (Z.n == 0) return Z.maxr;
    int cap = Z.outside;
    for (int z = 0; z < Z.n; ++z) {
        double d2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double t = __dadd_rn(x[d], -Z.c[z][d]);
            d2 = __dadd_rn(d2, __dmul_rn(t, t));
        }
        if (d2 >= Z.r2in[z] && d2 < Z.r2out[z]) cap = max(cap, Z.level[z]);
    }
    return cap;
}

__global__ void k_geom(int D, int Nv, int Nvp, const int* __restrict__ level, const int* __restrict__ base,
                       const uint32_t* __restrict__ key, int nb0, int nb1, int nb2, double vlo0, double vlo1,
                       double vlo2, double hb0, double hb1, double hb2, double* xi_d, double* w_d, float* xi_f,
                       float* w_f, float* xi_p, ZoneSet Z, int* ncap)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nvp) return;
    // pair layout: the d-th components of nodes 2j and 2j+1 side by side
    float* xp = xi_p + ((size_t)(k >> 1) * D) * 2 + (k & 1);
    if (k >= Nv) {
        for (int d = 0; d < D; ++d) {
            xi_d[(size_t)k * D + d] = 0.0;
            xi_f[(size_t)k * D + d] = 0.0f;
            xp[2 * d] = 0.0f;
        }
        w_d[k] = 0.0;
        w_f[k] = 0.0f;
        ncap[k] = 0;
        return;
    }
    double xc[3] = {0.0, 0.0, 0.0};
    const int nb[3] = {nb0, nb1, nb2};
    const double vlo[3] = {vlo0, vlo1, vlo2};
    const double hb[3] = {hb0, hb1, hb2};
    const int l = level[k];
    int b = base[k];
    const uint32_t kk = key[k];
    double wk = 1.0;
    for (int d = 0; d < D; ++d) {
        const int bi = b % nb[d];
        b /= nb[d];
        uint32_t o = 0;
        for (int m = 0; m < l; ++m) {
            const uint32_t digit = (kk >> (D * (l - 1 - m))) & ((1u << D) - 1u);
            o = 2u * o + ((digit >> d) & 1u);
        }
        const double frac = (double)(2u * o + 1u) / (double)(1u << (l + 1));
        const double x = __dadd_rn(vlo[d], __dmul_rn(hb[d], __dadd_rn((double)bi, frac)));
        xc[d] = x;
        xi_d[(size_t)k * D + d] = x;
        xi_f[(size_t)k * D + d] = (float)x;
        xp[2 * d] = (float)x;
        wk = __dmul_rn(wk, hb[d]);
    }
    const double wv = ldexp(wk, -D * l);
    w_d[k] = wv;
    w_f[k] = (float)wv;
    ncap[k] = zone_cap(Z, D, xc);
}

cudaError_t launch_geom(avs_ctx* c)
{
    const int n = c->Nvp;
    k_geom<<<(n + 255) / 256, 256, 0, c->stream>>>(c->D, c->Nv, c->Nvp, c->level, c->base, c->key, c->cfg.base[0],
                                                   c->cfg.base[1], c->cfg.base[2], c->cfg.vlo[0], c->cfg.vlo[1],
                                                   c->cfg.vlo[2], c->hb[0], c->hb[1], c->hb[2], c->xi_d, c->w_d,
                                                   c->xi_f, c->w_f, c->xi_p, c->zs, c->ncap);
    c->launches += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dt bound
// min over cells and nodes of |V_i| / sum_faces max(xi . An_out, 0)  (R5).
// Correctly rounded division is monotone in the divisor, so the minimum over
// the nodes of a cell equals |V_i| divided by the largest sum: one division per
// cell, bit-identical to dividing at every node.
//
// The largest FP64 sum is found without evaluating every node in FP64: an
// FP32 pass gives each node's sum S32 and a bound B on |S32 - S| (inputs and
// every operation rounded to FP32: |S32 - S| <= 11 u sum_j sum_d |xi_d A_jd|,
// u = 2^-24, while the results stay normal; B takes 32 u of that sum, formed as
// sum_d |xi_d| sum_j |A_jd|, plus 2^-100).  Only nodes with S32 + B >= max_k (S32 - B), which
// include the node of the exact maximum, are evaluated in FP64.
template <int NS>
__global__ void __launch_bounds__(128) k_dt_unit(int D, int Nv, const double* __restrict__ xi,
                                                 const float* __restrict__ xi_f, const int* __restrict__ slot,
                                                 const unsigned char* __restrict__ nslot,
                                                 const double* __restrict__ An, const float* __restrict__ An_f,
                                                 const double* __restrict__ vol, unsigned long long* out)
{
    __shared__ float wlo[4];
    __shared__ double wbig[4];
    const int i = blockIdx.x;
    const int ns = nslot[i];
    float A[NS][3];
    int fidx[NS];
    bool isR[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int sl = s < ns ? slot[i * AVS_MAXS + s] : -1;
        fidx[s] = sl >> 1;
        isR[s] = sl >= 0 && (sl & 1);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float a = (sl >= 0 && d < D) ? An_f[(size_t)fidx[s] * D + d] : 0.0f;
            A[s][d] = isR[s] ? -a : a;
        }
    }
    // sum_j sum_d |xi_d A_jd| = sum_d |xi_d| sum_j |A_jd|: the face sums once per cell
    float As[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        As[d] = 0.0f;
#pragma unroll
        for (int s = 0; s < NS; ++s) As[d] += fabsf(A[s][d]);
    }
    auto s32 = [&](int k, float& S, float& B) {
        float x[3] = {0.0f, 0.0f, 0.0f};
        for (int d = 0; d < D; ++d) x[d] = xi_f[(size_t)k * D + d];
        S = 0.0f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float sn = x[0] * A[s][0] + x[1] * A[s][1] + x[2] * A[s][2];
            S += sn > 0.0f ? sn : 0.0f;
        }
        B = (fabsf(x[0]) * As[0] + fabsf(x[1]) * As[1] + fabsf(x[2]) * As[2]) * 0x1p-19f + 0x1p-100f;
    };
    float lo = 0.0f;
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        float S, B;
        s32(k, S, B);
        lo = fmaxf(lo, S - B);
    }
    for (int o = 16; o > 0; o >>= 1) lo = fmaxf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    if ((threadIdx.x & 31) == 0) wlo[threadIdx.x >> 5] = lo;
    __syncthreads();
    lo = fmaxf(fmaxf(wlo[0], wlo[1]), fmaxf(wlo[2], wlo[3]));
    double big = 0.0;
    for (int k = threadIdx.x; k < Nv; k += blockDim.x) {
        float S, B;
        s32(k, S, B);
        if (S + B < lo) continue;
        const double* x = xi + (size_t)k * D;
        double sum = 0.0;
        for (int s = 0; s < ns; ++s) {
            const double* a = An + (size_t)fidx[s] * D;
            double sn = __dmul_rn(x[0], a[0]);
            for (int d = 1; d < D; ++d) sn = __dadd_rn(sn, __dmul_rn(x[d], a[d]));
            if (isR[s]) sn = -sn;
            if (sn > 0.0) sum = __dadd_rn(sum, sn);
        }
        big = sum > big ? sum : big;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, big, o);
        big = v > big ? v : big;
    }
    if ((threadIdx.x & 31) == 0) wbig[threadIdx.x >> 5] = big;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 4; ++w) big = wbig[w] > big ? wbig[w] : big;
        if (big > 0.0) atomicMin(out, dkey(__ddiv_rn(vol[i], big)));
    }
}

cudaError_t launch_dt_unit(avs_ctx* c)
{
    const unsigned long long init = ~0ull;
    cudaError_t e = cudaMemcpyAsync(c->dt_key, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    if (c->max_ns <= 4)
        k_dt_unit<4><<<c->Nc, 128, 0, c->stream>>>(c->D, c->Nv, c->xi_d, c->xi_f, c->slot, c->nslot, c->An_d,
                                                   c->An_f, c->vol, c->dt_key);
    else
        k_dt_unit<AVS_MAXS><<<c->Nc, 128, 0, c->stream>>>(c->D, c->Nv, c->xi_d, c->xi_f, c->slot, c->nslot,
                                                          c->An_d, c->An_f, c->vol, c->dt_key);
    c->launches += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ initial field
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// standard normal from SplitMix64 (Steele, Lea, Flood 2014) and Box-Muller
__device__ __forceinline__ double normal_ik(uint64_t seed, uint64_t i, uint64_t k)
{
    const uint64_t key = (i << 32) | k;
    const uint64_t u1 = splitmix64(seed ^ splitmix64(2u * key));
    const uint64_t u2 = splitmix64(seed ^ splitmix64(2u * key + 1u));
    const double U1 = ((double)(u1 >> 11) + 1.0) * 0x1p-53;
    const double U2 = (double)(u2 >> 11) * 0x1p-53;
    return sqrt(-2.0 * log(U1)) * cos(2.0 * AVS_PI * U2);
}

// Per-cell factors of the Maxwellian start, formed once per block by thread 0
// (an FP64 pow in every thread costs more than the block's node work).
struct MaxwellC {
    double pref, twoRT, U[3];    // rho / (2 pi R T)^(D/2), 2 R T, U
    float pref32, i2RT32, U32[3];
};

__device__ __forceinline__ void maxwell_consts(int D, double rho, const double* U, double RT, MaxwellC& m)
{
    m.pref = rho / pow(2.0 * AVS_PI * RT, 0.5 * D);
    m.twoRT = 2.0 * RT;
    m.pref32 = (float)m.pref;
    m.i2RT32 = (float)(1.0 / (2.0 * RT));
    for (int d = 0; d < 3; ++d) {
        m.U[d] = d < D ? U[d] : 0.0;
        m.U32[d] = (float)m.U[d];
    }
}

// g^eq at node k: FP64 (as the oracle) in the FP64 form; FP32 in the mixed
// form, whose f is stored in FP32 (expf, a few ulp of FP32 at most).  The
// noise factor 1 + amp z_ik uses the FP64 SplitMix64/Box-Muller normal in both.
template <typename T>
__device__ __forceinline__ double maxwell_node(int D, const MaxwellC& m, const double* __restrict__ xi,
                                               const float* __restrict__ xi32, int k, double amp, uint64_t seed,
                                               int i)
{
    if (sizeof(T) == 8) {
        double c2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double c = __dsub_rn(xi[(size_t)k * D + d], m.U[d]);
            c2 = __dadd_rn(c2, __dmul_rn(c, c));
        }
        double g = m.pref * exp(-c2 / m.twoRT);
        if (amp != 0.0) g *= 1.0 + amp * normal_ik(seed, (uint64_t)i, (uint64_t)k);
        return g;
    }
    float c2 = 0.0f;
    for (int d = 0; d < D; ++d) {
        const float c = xi32[(size_t)k * D + d] - m.U32[d];
        c2 += c * c;
    }
    float g = m.pref32 * expf(-c2 * m.i2RT32);
    if (amp != 0.0) g *= (float)(1.0 + amp * normal_ik(seed, (uint64_t)i, (uint64_t)k));
    return (double)g;
}

// f = g^eq(W_p) (1 + amp z_ik) per cell and node, pads zero; one block per cell.
template <typename T>
__global__ void __launch_bounds__(256) k_maxwell(int D, int NA, int Nv, int Nvp, const double* __restrict__ xi,
                                                 const float* __restrict__ xi32, const double* __restrict__ Wp,
                                                 double R, double amp, uint64_t seed, T* f)
{
    __shared__ MaxwellC m;
    __shared__ T h0;
    const int i = blockIdx.x;
    T* fi = f + (size_t)i * NA * Nvp;
    if (threadIdx.x == 0) {
        const double* P = Wp + (size_t)i * (D + 2);
        const double RT = R * P[D + 1];
        maxwell_consts(D, P[0], P + 1, RT, m);
        h0 = (T)((3 - D) * RT);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < Nvp; k += blockDim.x) {
        if (k >= Nv) {
            for (int a = 0; a < NA; ++a) fi[(size_t)a * Nvp + k] = T(0);
            continue;
        }
        const T G = (T)maxwell_node<T>(D, m, xi, xi32, k, amp, seed, i);
        fi[k] = G;
        if (NA == 2) fi[Nvp + k] = h0 * G;
    }
}

// Rykov model: G = g^eq(rho, U, T_t)(1 + amp z_ik), H = (3 - D) R T_t G,
// R = R T_r G from Wp = (rho, U, T_t, T_r).
template <typename T>
__global__ void __launch_bounds__(256) k_maxwell_rk(int D, int NA, int Nv, int Nvp, const double* __restrict__ xi,
                                                    const float* __restrict__ xi32, const double* __restrict__ Wp,
                                                    double R, double amp, uint64_t seed, T* f)
{
    __shared__ MaxwellC m;
    __shared__ double RTt_s, RTr_s;
    const int i = blockIdx.x;
    T* fi = f + (size_t)i * NA * Nvp;
    if (threadIdx.x == 0) {
        const double* P = Wp + (size_t)i * (D + 3);
        RTt_s = R * P[D + 1];
        RTr_s = R * P[D + 2];
        maxwell_consts(D, P[0], P + 1, RTt_s, m);
    }
    __syncthreads();
    const double RTt = RTt_s, RTr = RTr_s;
    const T h0 = (T)((3 - D) * RTt), r0 = (T)RTr;
    for (int k = threadIdx.x; k < Nvp; k += blockDim.x) {
        if (k >= Nv) {
            for (int a = 0; a < NA; ++a) fi[(size_t)a * Nvp + k] = T(0);
            continue;
        }
        const double g = maxwell_node<T>(D, m, xi, xi32, k, amp, seed, i);
        if (sizeof(T) == 8) {
            fi[k] = (T)g;
            if (D == 2) fi[Nvp + k] = (T)((3 - D) * RTt * g);
            fi[(size_t)(NA - 1) * Nvp + k] = (T)(RTr * g);
        } else {
            const T G = (T)g;
            fi[k] = G;
            if (D == 2) fi[Nvp + k] = h0 * G;
            fi[(size_t)(NA - 1) * Nvp + k] = r0 * G;
        }
    }
}

cudaError_t launch_maxwell(avs_ctx* c, const double* Wp, int Ncells, double amp, uint64_t seed, void* fout,
                           int f_is_double, int Nvp)
{
    if (c->model == AVS_RYKOV) {
        if (f_is_double || !c->mixed)
            k_maxwell_rk<double><<<Ncells, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, c->xi_d, c->xi_f, Wp,
                                                                c->cfg.R, amp, seed, (double*)fout);
        else
            k_maxwell_rk<float><<<Ncells, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, c->xi_d, c->xi_f, Wp,
                                                               c->cfg.R, amp, seed, (float*)fout);
        c->launches += 1;
        return cudaGetLastError();
    }
    if (f_is_double || !c->mixed)
        k_maxwell<double><<<Ncells, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, c->xi_d, c->xi_f, Wp, c->cfg.R, amp,
                                                         seed, (double*)fout);
    else
        k_maxwell<float><<<Ncells, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, c->xi_d, c->xi_f, Wp, c->cfg.R, amp,
                                                        seed, (float*)fout);
    c->launches += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ moments
// Conserved moments (Eq. 7) and heat flux (Eq. 8) of every cell, summed about
// the cell's carried velocity (when given) to limit cancellation: raw moments
// by one block per cell (FP32 partials, FP64 across warps), then the FP64
// conversion by one thread per cell.
template <typename T>
__device__ __forceinline__ void ref_velocity(int D, const double* Wref, int i, double* Vr)
{
    const int NW = D + 2;
    for (int d = 0; d < 3; ++d) Vr[d] = 0.0;
    if (Wref && Wref[(size_t)i * NW] > 0.0)
        for (int d = 0; d < D; ++d) Vr[d] = (double)(T)(Wref[(size_t)i * NW + 1 + d] / Wref[(size_t)i * NW]);
}

// Per-thread raw moments of the row fi about Vt (16-byte vectors of nodes per
// thread, thread t owns nodes tV.., tV + NT V..), returned as doubles: FP64
// sums in the FP64 form; compensated FP32 sums (about twice the FP32
// precision) in the mixed form, whose products w f x.. are FP32 as stored.
template <int D, typename T, int NT>
__device__ __forceinline__ void cell_raw_sums(int Nv, int Nvp, const T* __restrict__ fi, const T* __restrict__ xi,
                                              const T* __restrict__ w, const T* Vt, double* out)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v;
    constexpr int V = 16 / sizeof(T);
    T acc[NM], cmp[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = cmp[m] = T(0);
    for (int k0 = threadIdx.x * V; k0 < Nv; k0 += NT * V) {
        T x[V * D], wv[V], f0[V], f1[V];
        vload<T, V * D>(xi + (size_t)k0 * D, x);
        vload<T, V>(w + k0, wv);
        vload<T, V>(fi + k0, f0);
        if (NA == 2) vload<T, V>(fi + Nvp + k0, f1);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            T xs[D];
#pragma unroll
            for (int d = 0; d < D; ++d) xs[d] = x[v * D + d] - Vt[d];
            if constexpr (sizeof(T) == 4)
                raw_acc_c<D>(acc, cmp, xs, wv[v] * f0[v], NA == 2 ? wv[v] * f1[v] : T(0));
            else
                raw_acc<D>(acc, xs, wv[v] * f0[v], NA == 2 ? wv[v] * f1[v] : T(0));
        }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) out[m] = to_double(acc[m]) + to_double(cmp[m]);
}

template <int D, typename T, int NT>
__global__ void __launch_bounds__(NT) k_cell_moments(int Nv, int Nvp, const T* __restrict__ f,
                                                     const T* __restrict__ xi, const T* __restrict__ w,
                                                     const double* __restrict__ Wref, double* rmom)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v;
    __shared__ double sw[(NT / 32) * NM];
    __shared__ double mom[NM];
    const int i = blockIdx.x;
    double Vr[3];
    ref_velocity<T>(D, Wref, i, Vr);
    T Vt[D];
    for (int d = 0; d < D; ++d) Vt[d] = (T)Vr[d];
    const T* fi = f + (size_t)i * NA * Nvp;
    double acc[NM];
    cell_raw_sums<D, T, NT>(Nv, Nvp, fi, xi, w, Vt, acc);
    block_sum<NM, NT>(acc, sw, mom);
    if (threadIdx.x < NM) rmom[(size_t)i * NM + threadIdx.x] = mom[threadIdx.x];
}

template <int D, typename T>
__global__ void k_moments_finish(int Ncells, const double* __restrict__ rmom, const double* __restrict__ Wref,
                                 double* Wc, double* q)
{
    constexpr int NM = NMom<D>::v, NW = D + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ncells) return;
    double Vr[3], m[NM], W[5], qq[3];
    ref_velocity<T>(D, Wref, i, Vr);
    for (int k = 0; k < NM; ++k) m[k] = rmom[(size_t)i * NM + k];
    moments_from_raw<D>(m, Vr, W, q ? qq : nullptr, nullptr, nullptr);
    if (Wc)
        for (int k = 0; k < NW; ++k) Wc[(size_t)i * NW + k] = W[k];
    if (q)
        for (int d = 0; d < D; ++d) q[(size_t)i * D + d] = qq[d];
}

template <int D, typename T>
static cudaError_t cell_moments_t(avs_ctx* c, const T* f, const T* xi, const T* w, int Ncells, int Nvp,
                                  const double* Wref, double* Wc, double* q)
{
    k_cell_moments<D, T, 128><<<Ncells, 128, 0, c->stream>>>(c->Nv, Nvp, f, xi, w, Wref, c->rmom);
    k_moments_finish<D, T><<<(Ncells + 127) / 128, 128, 0, c->stream>>>(Ncells, c->rmom, Wref, Wc, q);
    c->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_cell_moments(avs_ctx* c, const void* f, int f_is_double, int Ncells, int Nvp, double* Wc_out,
                                double* q_out)
{
    if (c->model == AVS_RYKOV) return rk_launch_moments(c, f, f_is_double, Ncells, Nvp, Wc_out, q_out);
    const bool dbl = f_is_double || !c->mixed;
    const double* Wref = (Ncells == c->Nc) ? c->W[c->wcur] : nullptr;
    if (c->D == 2)
        return dbl ? cell_moments_t<2, double>(c, (const double*)f, c->xi_d, c->w_d, Ncells, Nvp, Wref, Wc_out, q_out)
                   : cell_moments_t<2, float>(c, (const float*)f, c->xi_f, c->w_f, Ncells, Nvp, Wref, Wc_out, q_out);
    return dbl ? cell_moments_t<3, double>(c, (const double*)f, c->xi_d, c->w_d, Ncells, Nvp, Wref, Wc_out, q_out)
               : cell_moments_t<3, float>(c, (const float*)f, c->xi_f, c->w_f, Ncells, Nvp, Wref, Wc_out, q_out);
}

// ------------------------------------------------------------------ criterion
// Per-cell inputs of the criterion, in the fixed order of the definition:
// rho, U_d = m_d / rho, e_int = rho E - 0.5 (sum m_d m_d) / rho.  The FP32
// screening form holds 1/rho, U_d, 0.5/e_int rounded to FP32.
__global__ void k_crit_cells(int D, int NW, int Ncells, const double* __restrict__ Wc, double* cp, float* cp32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ncells) return;
    const double* W = Wc + (size_t)i * NW;
    const double rho = W[0];
    double mm = 0.0;
    float* c32 = cp32 + (size_t)i * 8;
    for (int d = 0; d < 3; ++d) c32[1 + d] = 0.0f;
    for (int d = 0; d < D; ++d) {
        const double U = __ddiv_rn(W[1 + d], rho);
        cp[(size_t)i * 5 + 1 + d] = U;
        c32[1 + d] = (float)U;
        mm = __dadd_rn(mm, __dmul_rn(W[1 + d], W[1 + d]));
    }
    const double e = __dsub_rn(W[D + 1], __ddiv_rn(__dmul_rn(0.5, mm), rho));
    cp[(size_t)i * 5 + 0] = rho;
    cp[(size_t)i * 5 + 4] = e;
    c32[0] = 1.0f / (float)rho;
    c32[4] = 0.5f / (float)e;
}

__global__ void k_fill_key(unsigned long long* k, int n, unsigned long long v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = v;
}

__global__ void k_fill_u32(unsigned* k, int n, unsigned v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = v;
}

// ordered 32-bit key of a float (monotone for all non-NaN values)
__device__ __forceinline__ unsigned fkey(float x)
{
    const unsigned b = __float_as_uint(x);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) { return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k); }

__device__ __forceinline__ bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
__device__ __forceinline__ bool same_bits(double a, double b)
{
    return __double_as_longlong(a) == __double_as_longlong(b);
}

// Pass 1: per node, the largest lower bound max_i (m32 - B) over the cells.
template <typename T>
__global__ void k_crit_screen(int D, int NA, int Nv, int Nvp, int ncells, int cells_per_block,
                              const T* __restrict__ f, const float* __restrict__ xi, const float* __restrict__ w,
                              const float* __restrict__ cp32, const int* __restrict__ cells, unsigned* Mlo,
                              unsigned* Mhi)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const int j0 = blockIdx.y * cells_per_block;
    const int j1 = min(ncells, j0 + cells_per_block);
    float x[3];
    for (int d = 0; d < D; ++d) x[d] = xi[(size_t)k * D + d];
    const float wk = w[k];
    float lo = -INFINITY, hi = -INFINITY;
    for (int j = j0; j < j1; ++j) {
        const int i = cells ? cells[j] : j;
        float m, B;
        crit32(D, crit_scaled(f[(size_t)i * NA * Nvp + k]), wk, x, cp32 + (size_t)i * 8, m, B);
        lo = fmaxf(lo, m - B);
        hi = fmaxf(hi, m + B);
        if (m != m) hi = INFINITY;         // undecidable pair: force the exact evaluation
    }
    if (lo > -INFINITY) atomicMax(Mlo + k, fkey(lo));
    if (hi > -INFINITY) atomicMax(Mhi + k, fkey(hi));
}

// Pass 2: M_k = max over cells of max(M1, M2): M1 = (w G) / rho,
// M2 = ((0.5 (w G)) c^2) / e_int, c^2 summed left to right (Sec. 3.4, R9),
// in FP64 at the (cell, node) pairs whose screening interval reaches the
// node's lower bound: the pair of the exact maximum is always among them.
// With `decide`, only the split and merge tests of the marks are needed: a
// node whose interval [lo, hi] of s M_k lies clear of C1 and C2 (by 2^-20
// relative) is left to k_decode_M, which stores lo as its value; the tests
// give the same answers for it as for the exact M_k.
template <typename T>
__global__ void k_criterion(int D, int NA, int Nv, int Nvp, int ncells, int cells_per_block, const T* __restrict__ f,
                            const double* __restrict__ xi, const double* __restrict__ w, const double* __restrict__ cp,
                            const float* __restrict__ xi32, const float* __restrict__ w32,
                            const float* __restrict__ cp32, const unsigned* __restrict__ Mlo,
                            const unsigned* __restrict__ Mhi, int decide, float s32, float C1s, float C2s,
                            const int* __restrict__ cells, unsigned long long* Mkey)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    if (decide) {
        constexpr float eps = 0x1p-20f;
        const float slo = s32 * fkey_inv(Mlo[k]), shi = s32 * fkey_inv(Mhi[k]);
        const bool c1 = slo > C1s * (1.0f + eps) || shi < C1s * (1.0f - eps);
        const bool c2 = slo > C2s * (1.0f + eps) || shi < C2s * (1.0f - eps);
        if (c1 && c2) return;
    }
    const int j0 = blockIdx.y * cells_per_block;
    const int j1 = min(ncells, j0 + cells_per_block);
    double x[3];
    float xf[3];
    for (int d = 0; d < D; ++d) {
        x[d] = xi[(size_t)k * D + d];
        xf[d] = xi32[(size_t)k * D + d];
    }
    const double wk = w[k];
    const float wkf = w32[k];
    const float lo = fkey_inv(Mlo[k]);
    double best = -INFINITY;
    // a candidate whose inputs (f value and per-cell row) equal, bit for bit,
    // those of the last one evaluated has the same value: skip it (uniform
    // regions make many cells identical)
    int pi = -1;
    T Gp = T(0);
    for (int j = j0; j < j1; ++j) {
        const int i = cells ? cells[j] : j;
        const T Gt = f[(size_t)i * NA * Nvp + k];
        float m32, B;
        const float* c32 = cp32 + (size_t)i * 8;
        crit32(D, crit_scaled(Gt), wkf, xf, c32, m32, B);
        if (m32 + B < lo) continue;
        if (Gt == T(0) && c32[0] > 0.0f && c32[0] < INFINITY && c32[4] > 0.0f && c32[4] < INFINITY) {
            // G = +-0 with rho, e_int > 0: M1 = M2 = G exactly
            const double z = (double)Gt;
            best = z > best ? z : best;
            continue;
        }
        const double* p = cp + (size_t)i * 5;
        if (pi >= 0 && same_bits(Gt, Gp)) {
            const double* q = cp + (size_t)pi * 5;
            bool same = true;
#pragma unroll
            for (int c = 0; c < 5; ++c) same = same && __double_as_longlong(p[c]) == __double_as_longlong(q[c]);
            if (same) continue;
        }
        pi = i;
        Gp = Gt;
        const double G = (double)Gt;
        const double wg = __dmul_rn(wk, G);
        const double m1 = __ddiv_rn(wg, p[0]);
        double c2 = 0.0;
        for (int d = 0; d < D; ++d) {
            const double cc = __dsub_rn(x[d], p[1 + d]);
            c2 = __dadd_rn(c2, __dmul_rn(cc, cc));
        }
        const double m2 = __ddiv_rn(__dmul_rn(__dmul_rn(0.5, wg), c2), p[4]);
        const double mk = m1 > m2 ? m1 : m2;
        best = mk > best ? mk : best;
    }
    if (best > -INFINITY) atomicMax(Mkey + k, dkey(best));
}

// M_k from the exact maximum, or, for a node the decisions-only pass left
// out, the lower end of its screening interval (unscaled)
__global__ void k_decode_M(const unsigned long long* __restrict__ Mkey, const unsigned* __restrict__ Mlo, int decide,
                           double* M, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long key = Mkey[i];
    M[i] = (decide && key == dkey(-INFINITY)) ? (double)fkey_inv(Mlo[i]) * 0x1p-64 : dkey_inv(key);
}

cudaError_t launch_criterion(avs_ctx* c, const void* f, int f_is_double, int Ncells, int Nvp, const double* Wc,
                             const int* cells, int ncells_list, int decide)
{
    double* cp = c->crit_cp;
    k_crit_cells<<<(Ncells + 255) / 256, 256, 0, c->stream>>>(c->D, c->NW, Ncells, Wc, cp, c->crit_cp32);
    const unsigned long long ninf = dkey(-INFINITY);
    k_fill_key<<<(c->Nv + 255) / 256, 256, 0, c->stream>>>(c->Mkey, c->Nv, ninf);
    k_fill_u32<<<(c->Nv + 255) / 256, 256, 0, c->stream>>>(c->Mlo, c->Nv, 0x007fffffu);   // key of -inf
    k_fill_u32<<<(c->Nv + 255) / 256, 256, 0, c->stream>>>(c->Mhi, c->Nv, 0x007fffffu);
    const int n = cells ? ncells_list : Ncells;
    const int cpb = 64;
    dim3 g((c->Nv + 255) / 256, (n + cpb - 1) / cpb);
    const bool dbl = f_is_double || !c->mixed;
    const float s32 = (float)c->s_norm, C1s = (float)c->cfg.C1 * kCritScale, C2s = (float)c->cfg.C2 * kCritScale;
    if (n > 0) {
        if (dbl) {
            k_crit_screen<double><<<g, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, n, cpb, (const double*)f,
                                                            c->xi_f, c->w_f, c->crit_cp32, cells, c->Mlo, c->Mhi);
            k_criterion<double><<<g, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, n, cpb, (const double*)f, c->xi_d,
                                                          c->w_d, cp, c->xi_f, c->w_f, c->crit_cp32, c->Mlo, c->Mhi,
                                                          decide, s32, C1s, C2s, cells, c->Mkey);
        } else {
            k_crit_screen<float><<<g, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, n, cpb, (const float*)f,
                                                           c->xi_f, c->w_f, c->crit_cp32, cells, c->Mlo, c->Mhi);
            k_criterion<float><<<g, 256, 0, c->stream>>>(c->D, c->NA, c->Nv, Nvp, n, cpb, (const float*)f, c->xi_d,
                                                         c->w_d, cp, c->xi_f, c->w_f, c->crit_cp32, c->Mlo, c->Mhi,
                                                         decide, s32, C1s, C2s, cells, c->Mkey);
        }
    }
    k_decode_M<<<(c->Nv + 255) / 256, 256, 0, c->stream>>>(c->Mkey, c->Mlo, decide && n > 0, c->M, c->Nv);
    c->launches += (n > 0) ? 7 : 5;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ marks, scan, new tree
// emit[k] = number of new leaves produced by old leaf k; kind of the first:
// a group start (2^D sibling leaves, all s*M < C2, level >= 1) emits the
// parent; the other members of its group emit nothing; a leaf with
// s*M > C1 below the level cap emits its 2^D children; others emit themselves.
__global__ void k_group_start(int D, int Nv, const int* __restrict__ level, const int* __restrict__ base,
                              const uint32_t* __restrict__ key, const double* __restrict__ M, double s, double C2,
                              int uniform, int* gs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const int nch = 1 << D;
    int g = 0;
    if (!uniform && level[k] >= 1 && (key[k] & (uint32_t)(nch - 1)) == 0u && k + nch <= Nv) {
        g = 1;
        for (int c = 0; c < nch; ++c) {
            const int kk = k + c;
            if (level[kk] != level[k] || base[kk] != base[k] || key[kk] != key[k] + (uint32_t)c ||
                !(__dmul_rn(s, M[kk]) < C2))
                g = 0;
        }
    }
    gs[k] = g;
}

__global__ void k_emit(int D, int Nv, const int* __restrict__ level, const uint32_t* __restrict__ key,
                       const double* __restrict__ M, const int* __restrict__ gs, double s, double C1,
                       const int* __restrict__ ncap, int uniform, int* emit)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const int nch = 1 << D;
    int e;
    if (gs[k]) {
        e = 1;
    } else {
        const int dig = (int)(key[k] & (uint32_t)(nch - 1));
        const int st = k - dig;
        if (level[k] >= 1 && dig != 0 && st >= 0 && gs[st]) e = 0;
        else if (uniform || (__dmul_rn(s, M[k]) > C1 && level[k] < ncap[k])) e = nch;
        else e = 1;
    }
    emit[k] = e;
}

// Single-block exclusive scan (1024 threads, contiguous segments per thread,
// warp-shuffle scans); writes the total to *count.
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, int* out, int n, int* count)
{
    __shared__ int wsum[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (n + 1023) / 1024;
    const int b = min(n, t * per), e = min(n, b + per);
    int local = 0;
    for (int k = b; k < e; ++k) local += in[k];
    int x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = x - local + (warp > 0 ? wsum[warp - 1] : 0);
    for (int k = b; k < e; ++k) {
        out[k] = run;
        run += in[k];
    }
    if (t == 1023) *count = run;
}

__global__ void k_build(int D, int Nv, const int* __restrict__ level, const int* __restrict__ base,
                        const uint32_t* __restrict__ key, const int* __restrict__ gs, const int* __restrict__ emit,
                        const int* __restrict__ idx, int cap, int* nl, int* nb, uint32_t* nk, int* src, int* kind,
                        int* counters)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const int e = emit[k];
    const int n = idx[k];
    if (e == 0 || n + e > cap) return;
    const int nch = 1 << D;
    if (gs[k]) {
        nl[n] = level[k] - 1;
        nb[n] = base[k];
        nk[n] = key[k] >> D;
        src[n] = k;
        kind[n] = 1;
        atomicAdd(counters + 1, 1);
    } else if (e == nch) {
        for (int c = 0; c < nch; ++c) {
            nl[n + c] = level[k] + 1;
            nb[n + c] = base[k];
            nk[n + c] = (key[k] << D) | (uint32_t)c;
            src[n + c] = k;
            kind[n + c] = 0;
        }
        atomicAdd(counters + 0, 1);
    } else {
        nl[n] = level[k];
        nb[n] = base[k];
        nk[n] = key[k];
        src[n] = k;
        kind[n] = 0;
    }
}

// uniform = 1: every leaf splits (step 2 of Sec. 3.5), M is not read.
cudaError_t launch_adapt_tree(avs_ctx* c, double C1, double C2, int uniform)
{
    const int n = c->Nv;
    const int g = (n + 255) / 256;
    int* gs = c->newidx + c->cap;    // second half of the index scratch
    k_group_start<<<g, 256, 0, c->stream>>>(c->D, n, c->level, c->base, c->key, c->M, c->s_norm, C2, uniform, gs);
    k_emit<<<g, 256, 0, c->stream>>>(c->D, n, c->level, c->key, c->M, gs, c->s_norm, C1, c->ncap, uniform,
                                     c->emit);
    k_scan<<<1, 1024, 0, c->stream>>>(c->emit, c->newidx, n, c->d_count);
    cudaMemsetAsync(c->d_count + 1, 0, 2 * sizeof(int), c->stream);
    k_build<<<g, 256, 0, c->stream>>>(c->D, n, c->level, c->base, c->key, gs, c->emit, c->newidx, c->cap, c->level2,
                                      c->base2, c->key2, c->src, c->kind, c->d_count + 1);
    c->launches += 4;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ remap
// Consanguinity (Sec. 3.2): child = parent; merged parent = pairwise mean.
template <typename T>
__global__ void k_remap(int D, int NA, int Nv_new, int Nvp_old, int Nvp_new, const int* __restrict__ src,
                        const int* __restrict__ kind, const T* __restrict__ fo, T* fn)
{
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    const int ia = blockIdx.x;              // cell * NA + array
    if (k >= Nvp_new) return;
    T* out = fn + (size_t)ia * Nvp_new;
    if (k >= Nv_new) {
        out[k] = T(0);
        return;
    }
    const T* in = fo + (size_t)ia * Nvp_old + src[k];
    T v;
    if (kind[k] == 0) v = in[0];
    else if (D == 2) v = ((in[0] + in[1]) + (in[2] + in[3])) * T(0.25);
    else v = (((in[0] + in[1]) + (in[2] + in[3])) + ((in[4] + in[5]) + (in[6] + in[7]))) * T(0.125);
    out[k] = v;
}

cudaError_t launch_remap(avs_ctx* c, const void* fold, int Nvp_old, void* fnew, int Nvp_new, int Nv_new)
{
    dim3 g(c->Nc * c->NA, (Nvp_new + 255) / 256);
    if (c->mixed)
        k_remap<float><<<g, 256, 0, c->stream>>>(c->D, c->NA, Nv_new, Nvp_old, Nvp_new, c->src, c->kind,
                                                 (const float*)fold, (float*)fnew);
    else
        k_remap<double><<<g, 256, 0, c->stream>>>(c->D, c->NA, Nv_new, Nvp_old, Nvp_new, c->src, c->kind,
                                                  (const double*)fold, (double*)fnew);
    c->launches += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ correction
// f <- f + g^eq(W) - g^eq(W'), W' = moments of f, `iters` passes (Sec. 3.3,
// R12); then the remaining relative gap, max over cells, into *gap_key.
template <int D, typename T, int NT>
__global__ void __launch_bounds__(NT) k_correct(int Nv, int Nvp, T* f, const T* __restrict__ xi,
                                                const T* __restrict__ w, const double* __restrict__ Wt, double R,
                                                int iters, unsigned long long* gap_key)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    constexpr int V = 16 / sizeof(T);
    __shared__ double sw[(NT / 32) * NM];
    __shared__ double mom[NM];
    __shared__ EqPar<T> ea, eb;
    __shared__ float ce[7];                   // mixed form: coefficients of g(W) - g(W') (see below)
    const int i = blockIdx.x;
    T* fi = f + (size_t)i * NA * Nvp;
    const double* Wi = Wt + (size_t)i * NW;
    double rho, U[3], RT;
    prim<D>(Wi, rho, U, RT);
    double Vr[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) Vr[d] = (double)(T)U[d];
    T Vt[D];
    for (int d = 0; d < D; ++d) Vt[d] = (T)Vr[d];
    if (threadIdx.x == 0) ea = make_eq<D, T>(rho, U, RT, nullptr, 0.0);
    for (int it = 0; it <= iters; ++it) {
        // moments of the current f' (nodes per thread as in the update below)
        double acc[NM];
        cell_raw_sums<D, T, NT>(Nv, Nvp, fi, xi, w, Vt, acc);
        block_sum<NM, NT>(acc, sw, mom);
        if (it == iters) {
            if (threadIdx.x == 0) {
                double Wp[5];
                moments_from_raw<D>(mom, Vr, Wp, nullptr, nullptr, nullptr);
                double mref = 0.0;
                for (int d = 0; d < D; ++d) mref += Wi[1 + d] * Wi[1 + d];
                mref = sqrt(mref) + rho * sqrt(2.0 * RT);
                double e = fabs(Wp[0] - Wi[0]) / fabs(Wi[0]);
                for (int d = 0; d < D; ++d) e = fmax(e, fabs(Wp[1 + d] - Wi[1 + d]) / mref);
                e = fmax(e, fabs(Wp[D + 1] - Wi[D + 1]) / fabs(Wi[D + 1]));
                if (e != e) e = INFINITY;
                atomicMax(gap_key, dkey(e));
            }
            break;
        }
        if (threadIdx.x == 0) {
            double Wp[5], rp, Up[3], RTp;
            moments_from_raw<D>(mom, Vr, Wp, nullptr, nullptr, nullptr);
            prim<D>(Wp, rp, Up, RTp);
            eb = make_eq<D, T>(rp, Up, RTp, nullptr, 0.0);
            if constexpr (sizeof(T) == 4) {
                // g(W) - g(W') = g(W') expm1(E), E = log of the ratio of the two
                // Maxwellians = e0 + e1 . xi + e2 |xi|^2, coefficients in FP64
                // from the differences of the states (no cancellation), so the
                // FP32 difference is accurate where W' is close to W; H: the
                // same with (3 - D) R T (ratio and difference)
                const double a = 0.5 / RT;
                const double e2 = (RT - RTp) / (2.0 * RT * RTp);      // b - a
                double dU[3], sU[3], Ub2 = 0.0, dUs = 0.0;
                for (int d = 0; d < D; ++d) {
                    dU[d] = U[d] - Up[d];
                    sU[d] = U[d] + Up[d];
                    Ub2 += Up[d] * Up[d];
                    dUs += dU[d] * sU[d];
                }
                const double lnA = log1p((rho - rp) / rp) - 0.5 * D * log1p((RT - RTp) / RTp);
                ce[0] = (float)(lnA - a * dUs + e2 * Ub2);
                for (int d = 0; d < 3; ++d) ce[1 + d] = d < D ? (float)(2.0 * (a * dU[d] - e2 * Up[d])) : 0.0f;
                ce[4] = (float)e2;
                ce[5] = (float)((3 - D) * RT);
                ce[6] = (float)((3 - D) * (RT - RTp));
            }
        }
        __syncthreads();
        // f' <- f' + g(W) - g(W')  (Sec. 3.3)
        for (int k0 = threadIdx.x * V; k0 < Nv; k0 += NT * V) {
            T x[V * D], f0[V], f1[V];
            vload<T, V * D>(xi + (size_t)k0 * D, x);
            vload<T, V>(fi + k0, f0);
            if (NA == 2) vload<T, V>(fi + Nvp + k0, f1);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T dG, dH;
                if constexpr (sizeof(T) == 4) {
                    T gb, gbh;
                    eq_eval<D>(eb, x + v * D, gb, gbh);
                    const T* xv = x + v * D;
                    T E = ce[0], x2 = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        E += ce[1 + d] * xv[d];
                        x2 += xv[d] * xv[d];
                    }
                    E += ce[4] * x2;
                    const T em1 = expm1f(E);
                    dG = gb * em1;
                    dH = gb * (ce[5] * em1 + ce[6]);
                } else {
                    T ga, gah, gb, gbh;
                    eq_eval<D>(ea, x + v * D, ga, gah);
                    eq_eval<D>(eb, x + v * D, gb, gbh);
                    dG = ga - gb;
                    dH = gah - gbh;
                }
                const bool real = k0 + v < Nv;
                f0[v] = real ? f0[v] + dG : f0[v];
                if (NA == 2) f1[v] = real ? f1[v] + dH : f1[v];
            }
            vstore<T, V>(fi + k0, f0);
            if (NA == 2) vstore<T, V>(fi + Nvp + k0, f1);
        }
    }
}

cudaError_t launch_correct(avs_ctx* c, void* f, const double* Wtarget, int iters)
{
    if (c->model == AVS_RYKOV) return rk_launch_correct(c, f, Wtarget, iters);
    const unsigned long long zero = dkey(0.0);
    cudaError_t e = cudaMemcpyAsync(c->gap_d, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    unsigned long long* gk = (unsigned long long*)c->gap_d;
    if (c->D == 2) {
        if (c->mixed)
            k_correct<2, float, 128><<<c->Nc, 128, 0, c->stream>>>(c->Nv, c->Nvp, (float*)f, c->xi_f, c->w_f,
                                                                         Wtarget, c->cfg.R, iters, gk);
        else
            k_correct<2, double, 128><<<c->Nc, 128, 0, c->stream>>>(c->Nv, c->Nvp, (double*)f, c->xi_d,
                                                                          c->w_d, Wtarget, c->cfg.R, iters, gk);
    } else {
        if (c->mixed)
            k_correct<3, float, 128><<<c->Nc, 128, 0, c->stream>>>(c->Nv, c->Nvp, (float*)f, c->xi_f, c->w_f,
                                                                         Wtarget, c->cfg.R, iters, gk);
        else
            k_correct<3, double, 128><<<c->Nc, 128, 0, c->stream>>>(c->Nv, c->Nvp, (double*)f, c->xi_d,
                                                                          c->w_d, Wtarget, c->cfg.R, iters, gk);
    }
    c->launches += 1;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ conversions
template <typename T>
__global__ void k_to_double(int Nv, int Nvp, const T* __restrict__ f, double* out)
{
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    const int ia = blockIdx.x;
    if (k < Nv) out[(size_t)ia * Nv + k] = (double)f[(size_t)ia * Nvp + k];
}

template <typename T>
__global__ void k_from_double(int Nv, int Nvp, const double* __restrict__ in, T* f)
{
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    const int ia = blockIdx.x;
    if (k < Nvp) f[(size_t)ia * Nvp + k] = k < Nv ? (T)in[(size_t)ia * Nv + k] : T(0);
}

cudaError_t launch_to_double(avs_ctx* c, const void* f, double* out, int Nvp)
{
    dim3 g(c->Nc * c->NA, (c->Nv + 255) / 256);
    if (c->mixed) k_to_double<float><<<g, 256, 0, c->stream>>>(c->Nv, Nvp, (const float*)f, out);
    else k_to_double<double><<<g, 256, 0, c->stream>>>(c->Nv, Nvp, (const double*)f, out);
    c->launches += 1;
    return cudaGetLastError();
}

template <typename T>
__global__ void k_gather_double(int Nv, int Nvp, int NA, const T* __restrict__ f, const int* __restrict__ cells,
                                double* out)
{
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    const int ja = blockIdx.x;                      // (list entry, array)
    if (k >= Nv) return;
    const int j = ja / NA, a = ja % NA;
    out[(size_t)ja * Nv + k] = (double)f[((size_t)cells[j] * NA + a) * Nvp + k];
}

cudaError_t launch_gather_double(avs_ctx* c, const int* cells_d, int ncells, double* out)
{
    dim3 g(ncells * c->NA, (c->Nv + 255) / 256);
    if (c->mixed)
        k_gather_double<float><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->NA, (const float*)c->f[c->cur], cells_d,
                                                         out);
    else
        k_gather_double<double><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->NA, (const double*)c->f[c->cur],
                                                          cells_d, out);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_from_double(avs_ctx* c, const double* in, void* f, int Nvp)
{
    dim3 g(c->Nc * c->NA, (Nvp + 255) / 256);
    if (c->mixed) k_from_double<float><<<g, 256, 0, c->stream>>>(c->Nv, Nvp, in, (float*)f);
    else k_from_double<double><<<g, 256, 0, c->stream>>>(c->Nv, Nvp, in, (double*)f);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace avs
