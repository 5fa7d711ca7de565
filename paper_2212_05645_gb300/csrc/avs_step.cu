// One explicit UGKS step on the global velocity mesh (paper Sec. 2.3, with
// the explicit readings R1-R4), as four kernels.
//
// k_foot: one thread block per (cell, node chunk).  The limited
//   least-squares gradient L grad phi of the cell (Sec. 2.3.3: weights
//   1/|d|^2, Venkatakrishnan limiter with epsilon^2 = (K dx)^3 phi_C^2) at
//   each node, kept in registers, and the
//   foot values phi_C + (L grad phi)_C . (x_f - xi h - x_C) of every face of
//   the cell at the nodes where the cell is upwind (sign of xi . An), written
//   to the face's row: each face node gets its foot value exactly once.
//
// k_face: one thread block per face.  The raw velocity moments of the foot
//   values (interface W of Eq. w_interface and heat flux), the interface
//   Shakhov state (Eqs. 3, equ28, R4), then the interface distribution
//   phi_ij = tau/(tau+h) phi_bar + h/(tau+h) g_ij per node.  Writes the
//   per-node flux (xi . An) phi_ij over the foot values and the face's
//   area-weighted flux of W.  Boundaries: diffuse wall with zero net mass
//   flux, far-field Maxwellian (R8).
//
// k_cell_state / k_cell: one thread per cell, then one block per cell.
//   Lagged heat flux from the moments of f^n (R3), W~ = W - dt/|V| sum_j A F_j
//   (R2), the cell's Shakhov state and the collision update of every node
//   from the net flux of its faces (diagonal of Eq. SGS_phi, R1).
//
// Every face is evaluated once, so the two cells of a face see the same flux
// and W telescopes exactly.  f^n and W^n are read-only during the step; no
// block waits on another.  Sums: per-thread and warp sums in the element
// type, FP64 across warps and in every per-cell / per-face formula.  The
// limited-gradient kernel k_grad (gradients stored next to f) serves the
// Rykov model's face kernels.
#include <algorithm>
#include <type_traits>

#include "avs_dev.cuh"
#include "avs_internal.h"

namespace avs {

// nodes per thread per iteration: 16-byte vector loads along the node index
template <typename T> struct VW { static constexpr int v = 16 / sizeof(T); };

template <typename T, int V>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T* o)
{
    if constexpr (sizeof(T) == 4 && V == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    } else if constexpr (sizeof(T) == 4 && V == 2) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        o[0] = q.x; o[1] = q.y;
    } else if constexpr (sizeof(T) == 8 && V == 2) {
        const double2 q = *reinterpret_cast<const double2*>(p);
        o[0] = q.x; o[1] = q.y;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) o[v] = p[v];
    }
}

// ldv through L2 only (values this block reads once)
template <typename T, int V>
__device__ __forceinline__ void ldv_cg(const T* __restrict__ p, T* o)
{
    if constexpr (sizeof(T) == 4 && V == 4) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    } else if constexpr (sizeof(T) == 4 && V == 2) {
        const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = q.x; o[1] = q.y;
    } else if constexpr (sizeof(T) == 8 && V == 2) {
        const double2 q = __ldcg(reinterpret_cast<const double2*>(p));
        o[0] = q.x; o[1] = q.y;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) o[v] = __ldcg(p + v);
    }
}

template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const T* o)
{
    if constexpr (sizeof(T) == 4 && V == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(T) == 4 && V == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else if constexpr (sizeof(T) == 8 && V == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = o[v];
    }
}

// N consecutive elements (N * sizeof(T) a multiple of 16 bytes, 16-byte
// aligned) as 16-byte vector loads / stores.
template <typename T, int N>
__device__ __forceinline__ void ldvn(const T* __restrict__ p, T* o)
{
    constexpr int W = 16 / sizeof(T);
#pragma unroll
    for (int j = 0; j < N / W; ++j) ldv<T, W>(p + j * W, o + j * W);
}

template <typename T, int N>
__device__ __forceinline__ void stvn(T* p, const T* o)
{
    constexpr int W = 16 / sizeof(T);
#pragma unroll
    for (int j = 0; j < N / W; ++j) stv<T, W>(p + j * W, o + j * W);
}

// ------------------------------------------------------------------ k_grad
// G[i][a][d][k] = L * (grad phi)_d of array a of cell i at node k.  Each
// thread handles VG consecutive nodes (rows are padded to 32 nodes, so the
// vector stays inside the row) to keep more loads in flight.  NS: face slots
// unrolled (4 when every cell of a 2D mesh has at most 4 faces, else 6).
// NA: arrays per cell (2 or 1 for the monatomic gas, 3 or 2 for the Rykov model).
template <int D, typename T, int VG, int NS, int NA>
__global__ void __launch_bounds__(256) k_grad(int Nv, int Nvp, int limiter, const T* __restrict__ f,
                                              T* __restrict__ G, CellGeo<T> geo)
{
    static_assert((VG * sizeof(T)) % 16 == 0, "whole 16-byte vectors per thread");
    const int i = blockIdx.x;
    const int k0 = (blockIdx.y * blockDim.x + threadIdx.x) * VG;
    if (k0 >= Nv) return;
    const size_t cstride = (size_t)NA * Nvp;
    const int ns = geo.ns[i];
    // slots without a neighbour read the cell itself (difference 0) and have
    // zero weights and offsets, so they add nothing and need no branch
    int nb[NS];
    T cg[NS][D], rr[NS][D];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int n = s < ns ? geo.nbr[i * AVS_MAXS + s] : -1;
        nb[s] = n >= 0 ? n : i;
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
        T phi[VG], nv[NS][VG];
        ldvn<T, VG>(fa + (size_t)i * cstride, phi);
#pragma unroll
        for (int s = 0; s < NS; ++s) ldvn<T, VG>(fa + (size_t)nb[s] * cstride, nv[s]);
        T* o = G + ((size_t)i * NA + a) * D * Nvp + k0;
        T out[D][VG];
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            T g[D];
#pragma unroll
            for (int d = 0; d < D; ++d) g[d] = T(0);
            T dmax = T(0), dmin = T(0);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const T dd = nv[s][v] - phi[v];
#pragma unroll
                for (int d = 0; d < D; ++d) g[d] += cg[s][d] * dd;
                dmax = dd > dmax ? dd : dmax;
                dmin = dd < dmin ? dd : dmin;
            }
            T L = T(1);
            if (limiter == 1) {
                T p = T(0), n = T(0);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    T d2 = g[0] * rr[s][0];
#pragma unroll
                    for (int d = 1; d < D; ++d) d2 += g[d] * rr[s][d];
                    p = d2 > p ? d2 : p;
                    n = d2 < n ? d2 : n;
                }
                // epsilon^2 = (K dx)^3 phi_C^2: scaled to the limited value (R6)
                const T e2p = e2 * phi[v] * phi[v];
                if (p > T(0)) { const T t = venkat(dmax, p, e2p); L = t < L ? t : L; }
                if (n < T(0)) { const T t = venkat(dmin, n, e2p); L = t < L ? t : L; }
            }
#pragma unroll
            for (int d = 0; d < D; ++d) out[d][v] = L * g[d];
        }
#pragma unroll
        for (int d = 0; d < D; ++d) stvn<T, VG>(o + (size_t)d * Nvp, out[d]);
    }
}

// ------------------------------------------------------------------ k_foot
// Cell-centric reconstruction (Sec. 2.3.3).  Thread block (cell i, 256 x VG
// nodes): the limited gradient of every array of cell i (as k_grad, kept in
// registers), then for every face slot s of the cell the foot values
//   phi_bar = phi_i + (L grad phi)_i . (x_f - x_i - xi h)
// at the nodes where i is that face's upwind cell (xi . An >= 0 for the face's
// L cell, < 0 for its R cell; xi . An summed without contraction, the same
// value the face kernel tests), written to the face's row of
// FB [face][array][Nvp].  Every node of an interior face is written exactly
// once, by its upwind cell; of a boundary face only the outgoing half.  The
// gradient itself is never stored.
template <int D, typename T, int VG, int NS, int NA>
__global__ void __launch_bounds__(256) k_foot(int Nv, int Nvp, int limiter, T h, const T* __restrict__ f,
                                              T* __restrict__ FB, CellGeo<T> geo, const int* __restrict__ slot,
                                              const T* __restrict__ An, const T* __restrict__ xi)
{
    static_assert((VG * sizeof(T)) % 16 == 0, "whole 16-byte vectors per thread");
    const int i = blockIdx.x;
    const int k0 = (blockIdx.y * blockDim.x + threadIdx.x) * VG;
    if (k0 >= Nv) return;
    const size_t cstride = (size_t)NA * Nvp;
    const int ns = geo.ns[i];
    int nb[NS];
    T cg[NS][D], rr[NS][D];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int n = s < ns ? geo.nbr[i * AVS_MAXS + s] : -1;
        nb[s] = n >= 0 ? n : i;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            cg[s][d] = s < ns ? geo.cg[(size_t)(i * AVS_MAXS + s) * D + d] : T(0);
            rr[s][d] = s < ns ? geo.r[(size_t)(i * AVS_MAXS + s) * D + d] : T(0);
        }
    }
    const T e2 = geo.eps2[i];
    T phi[NA][VG], G[NA][D][VG];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const T* fa = f + (size_t)a * Nvp + k0;
        T nv[NS][VG];
        ldvn<T, VG>(fa + (size_t)i * cstride, phi[a]);
#pragma unroll
        for (int s = 0; s < NS; ++s) ldvn<T, VG>(fa + (size_t)nb[s] * cstride, nv[s]);
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            T g[D], dd[NS];
#pragma unroll
            for (int d = 0; d < D; ++d) g[d] = T(0);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                dd[s] = nv[s][v] - phi[a][v];
#pragma unroll
                for (int d = 0; d < D; ++d) g[d] += cg[s][d] * dd[s];
            }
            T L = T(1);
            if (limiter == 1) {
                // extremes of the neighbour differences and of the face
                // projections g . r_s (both include 0: the cell itself)
                T d2[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    d2[s] = g[0] * rr[s][0];
#pragma unroll
                    for (int d = 1; d < D; ++d) d2[s] += g[d] * rr[s][d];
                }
                T dmax, dmin, p, n;
                if constexpr (sizeof(T) == 4 && NS == 6) {
                    dmax = max3f(max3f(dd[0], dd[1], dd[2]), max3f(dd[3], dd[4], dd[5]), 0.0f);
                    dmin = min3f(min3f(dd[0], dd[1], dd[2]), min3f(dd[3], dd[4], dd[5]), 0.0f);
                    p = max3f(max3f(d2[0], d2[1], d2[2]), max3f(d2[3], d2[4], d2[5]), 0.0f);
                    n = min3f(min3f(d2[0], d2[1], d2[2]), min3f(d2[3], d2[4], d2[5]), 0.0f);
                } else if constexpr (sizeof(T) == 4 && NS == 4) {
                    dmax = max3f(max3f(dd[0], dd[1], dd[2]), dd[3], 0.0f);
                    dmin = min3f(min3f(dd[0], dd[1], dd[2]), dd[3], 0.0f);
                    p = max3f(max3f(d2[0], d2[1], d2[2]), d2[3], 0.0f);
                    n = min3f(min3f(d2[0], d2[1], d2[2]), d2[3], 0.0f);
                } else {
                    dmax = dmin = p = n = T(0);
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        dmax = dd[s] > dmax ? dd[s] : dmax;
                        dmin = dd[s] < dmin ? dd[s] : dmin;
                        p = d2[s] > p ? d2[s] : p;
                        n = d2[s] < n ? d2[s] : n;
                    }
                }
                // epsilon^2 = (K dx)^3 phi_C^2: scaled to the limited value (R6)
                const T e2p = e2 * phi[a][v] * phi[a][v];
                if (p > T(0)) { const T t = venkat(dmax, p, e2p); L = t < L ? t : L; }
                if (n < T(0)) { const T t = venkat(dmin, n, e2p); L = t < L ? t : L; }
            }
            if (limiter == 0) L = T(0);          // first order: phi_bar = phi_C
#pragma unroll
            for (int d = 0; d < D; ++d) G[a][d][v] = L * g[d];
        }
    }
    // node coordinates of the thread's nodes
    T x[VG][D];
    {
        T xx[VG * D];
        ldvn<T, VG * D>(xi + (size_t)k0 * D, xx);
#pragma unroll
        for (int v = 0; v < VG; ++v)
#pragma unroll
            for (int d = 0; d < D; ++d) x[v][d] = xx[v * D + d];
    }
    // phi_bar = A + G . r_s with A = phi - h G . xi, the part common to the faces
    T A[NA][VG];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            T gx = G[a][0][v] * x[v][0];
#pragma unroll
            for (int d = 1; d < D; ++d) gx += G[a][d][v] * x[v][d];
            A[a][v] = phi[a][v] - h * gx;
        }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (s >= ns) break;
        const int sl = slot[i * AVS_MAXS + s];
        const int fc = sl >> 1;
        const bool isR = sl & 1;
        T an[D];
#pragma unroll
        for (int d = 0; d < D; ++d) an[d] = An[(size_t)fc * D + d];
        bool up[VG];
        bool all = true, any = false;
#pragma unroll
        for (int v = 0; v < VG; ++v) {
            // the face kernel's xi . An (FP64: summed without contraction, so
            // the upwind choice is the plain sequential one; FP32: any fixed
            // formula, since only the face's two cells must agree)
            T sn;
            if constexpr (sizeof(T) == 8) {
                sn = dot_rn<D>(x[v], an);
            } else {
                sn = x[v][0] * an[0];
#pragma unroll
                for (int d = 1; d < D; ++d) sn = fmaf(x[v][d], an[d], sn);
            }
            up[v] = isR ? (sn < T(0)) : (sn >= T(0));
            all = all && up[v];
            any = any || up[v];
        }
        if (!any) continue;
        T* row = FB + (size_t)fc * NA * Nvp + k0;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            T out[VG];
#pragma unroll
            for (int v = 0; v < VG; ++v) {
                T val = A[a][v];
#pragma unroll
                for (int d = 0; d < D; ++d) val += G[a][d][v] * rr[s][d];
                out[v] = val;
            }
            if (all) {
                stvn<T, VG>(row + (size_t)a * Nvp, out);
            } else {
#pragma unroll
                for (int v = 0; v < VG; ++v)
                    if (up[v]) row[(size_t)a * Nvp + v] = out[v];
            }
        }
    }
}

// k_foot for the FP32 form in packed two-lane arithmetic: four nodes per
// thread as two pairs, each lane doing k_foot's operations (the same products
// and fused multiply-adds in the same order, so the same foot values; the
// limiter's two ratios are evaluated in both lanes and selected per lane).
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, bc2(-1.0f), a); }   // a - b, one rounding

template <int NS>
__device__ __forceinline__ void ext4(const float* v, float& mx, float& mn)
{
    if constexpr (NS == 6) {
        mx = max3f(max3f(v[0], v[1], v[2]), max3f(v[3], v[4], v[5]), 0.0f);
        mn = min3f(min3f(v[0], v[1], v[2]), min3f(v[3], v[4], v[5]), 0.0f);
    } else if constexpr (NS == 4) {
        mx = max3f(max3f(v[0], v[1], v[2]), v[3], 0.0f);
        mn = min3f(min3f(v[0], v[1], v[2]), v[3], 0.0f);
    } else {
        mx = mn = 0.0f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            mx = fmaxf(mx, v[s]);
            mn = fminf(mn, v[s]);
        }
    }
}

// Venkatakrishnan ratio of venkat() in two lanes (division as a reciprocal
// and a product, like fdiv); capped at 1
__device__ __forceinline__ float2 venkat2(float2 d1, float2 d2, float2 eps2)
{
    const float2 d11 = mul2(d1, d1);
    const float2 num = fma2(mul2(bc2(2.0f), d1), d2, add2(d11, eps2));
    const float2 den = add2(fma2(d1, d2, fma2(mul2(bc2(2.0f), d2), d2, d11)), eps2);
    const float2 v = make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
    return make_float2(v.x < 1.0f ? v.x : 1.0f, v.y < 1.0f ? v.y : 1.0f);
}

template <int D, int NS, int NA>
__global__ void __launch_bounds__(128, 8) k_foot_f2(int Nv, int Nvp, int limiter, float h, const float* __restrict__ f,
                                                 float* __restrict__ FB, CellGeo<float> geo,
                                                 const int* __restrict__ slot, const float* __restrict__ An,
                                                 const float* __restrict__ xp)
{
    constexpr int VG = 4;
    const int i = blockIdx.x;
    const int t = threadIdx.x;
    const int k0 = (blockIdx.y * blockDim.x + t) * VG;
    const int ns = geo.ns[i];
    // the cell's geometry, once per block: least-squares weights, face
    // offsets and face normals per slot (padded to four floats, read back as
    // one 16-byte vector), neighbour cells and slot codes
    __shared__ __align__(16) float gs[3][NS][4];
    __shared__ int gn[2][NS];
    if (t < NS * 4) {
        const int s = t >> 2, d = t & 3;
        const bool on = s < ns && d < D;
        gs[0][s][d] = on ? geo.cg[(size_t)(i * AVS_MAXS + s) * D + d] : 0.0f;
        gs[1][s][d] = on ? geo.r[(size_t)(i * AVS_MAXS + s) * D + d] : 0.0f;
    } else if (t >= 32 && t < 32 + NS) {
        const int s = t - 32;
        const int n = s < ns ? geo.nbr[i * AVS_MAXS + s] : -1;
        const int sl = s < ns ? slot[i * AVS_MAXS + s] : 0;
        gn[0][s] = n >= 0 ? n : i;
        gn[1][s] = sl;
#pragma unroll
        for (int d = 0; d < 4; ++d) gs[2][s][d] = (s < ns && d < D) ? An[(size_t)(sl >> 1) * D + d] : 0.0f;
    }
    __syncthreads();
    if (k0 >= Nv) return;
    const size_t cstride = (size_t)NA * Nvp;
    auto vec = [&](int q, int s, float (&o)[D]) {
        const float4 v = *reinterpret_cast<const float4*>(gs[q][s]);
        o[0] = v.x;
        o[1] = v.y;
        if constexpr (D == 3) o[2] = v.z;
    };
    const float e2 = geo.eps2[i];
    float2 phi[NA][2], G[NA][D][2];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const float* fa = f + (size_t)a * Nvp + k0;
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(fa + (size_t)i * cstride));
        phi[a][0] = lo2(c4);
        phi[a][1] = hi2(c4);
        float4 n4[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) n4[s] = __ldg(reinterpret_cast<const float4*>(fa + (size_t)gn[0][s] * cstride));
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float2 g[D], dd[NS];
#pragma unroll
            for (int d = 0; d < D; ++d) g[d] = bc2(0.0f);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                float cg[D];
                vec(0, s, cg);
                dd[s] = sub2(p ? hi2(n4[s]) : lo2(n4[s]), phi[a][p]);
#pragma unroll
                for (int d = 0; d < D; ++d) g[d] = fma2(bc2(cg[d]), dd[s], g[d]);
            }
            float2 L = bc2(1.0f);
            if (limiter == 1) {
                float2 d2[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    float rr[D];
                    vec(1, s, rr);
                    d2[s] = mul2(g[0], bc2(rr[0]));
#pragma unroll
                    for (int d = 1; d < D; ++d) d2[s] = fma2(g[d], bc2(rr[d]), d2[s]);
                }
                float dx[NS], dy[NS], ex[NS], ey[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    dx[s] = dd[s].x; dy[s] = dd[s].y;
                    ex[s] = d2[s].x; ey[s] = d2[s].y;
                }
                float2 dmax, dmin, pp, nn;
                ext4<NS>(dx, dmax.x, dmin.x);
                ext4<NS>(dy, dmax.y, dmin.y);
                ext4<NS>(ex, pp.x, nn.x);
                ext4<NS>(ey, pp.y, nn.y);
                // epsilon^2 = (K dx)^3 phi_C^2: scaled to the limited value (R6)
                const float2 e2p = mul2(mul2(bc2(e2), phi[a][p]), phi[a][p]);
                const float2 tp = venkat2(dmax, pp, e2p);
                const float2 tn = venkat2(dmin, nn, e2p);
                if (pp.x > 0.0f) L.x = tp.x;
                if (pp.y > 0.0f) L.y = tp.y;
                if (nn.x < 0.0f && tn.x < L.x) L.x = tn.x;
                if (nn.y < 0.0f && tn.y < L.y) L.y = tn.y;
            }
            if (limiter == 0) L = bc2(0.0f);     // first order: phi_bar = phi_C
#pragma unroll
            for (int d = 0; d < D; ++d) G[a][d][p] = mul2(L, g[d]);
        }
    }
    // node coordinates of the thread's nodes, as lane pairs (xp: the pair layout)
    float2 X[2][D];
    {
        float xx[VG * D];
        ldvn<float, VG * D>(xp + (size_t)k0 * D, xx);
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int d = 0; d < D; ++d) X[p][d] = make_float2(xx[(p * D + d) * 2], xx[(p * D + d) * 2 + 1]);
    }
    // phi_bar = A + G . r_s with A = phi - h G . xi, the part common to the faces
    float2 A[NA][2];
#pragma unroll
    for (int a = 0; a < NA; ++a)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float2 gx = mul2(G[a][0][p], X[p][0]);
#pragma unroll
            for (int d = 1; d < D; ++d) gx = fma2(G[a][d][p], X[p][d], gx);
            A[a][p] = fma2(bc2(-h), gx, phi[a][p]);
        }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (s >= ns) break;
        const int sl = gn[1][s];
        const int fc = sl >> 1;
        const bool isR = sl & 1;
        float an[D], rr[D];
        vec(2, s, an);
        vec(1, s, rr);
        bool up[4];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            // xi . An as in k_foot: a product, then fused multiply-adds
            float2 sn = mul2(X[p][0], bc2(an[0]));
#pragma unroll
            for (int d = 1; d < D; ++d) sn = fma2(X[p][d], bc2(an[d]), sn);
            up[2 * p] = isR ? (sn.x < 0.0f) : (sn.x >= 0.0f);
            up[2 * p + 1] = isR ? (sn.y < 0.0f) : (sn.y >= 0.0f);
        }
        const bool all = up[0] && up[1] && up[2] && up[3];
        const bool any = up[0] || up[1] || up[2] || up[3];
        if (!any) continue;
        float* row = FB + (size_t)fc * NA * Nvp + k0;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            float2 o[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float2 val = A[a][p];
#pragma unroll
                for (int d = 0; d < D; ++d) val = fma2(G[a][d][p], bc2(rr[d]), val);
                o[p] = val;
            }
            float* ra = row + (size_t)a * Nvp;
            if (all) {
                *reinterpret_cast<float4*>(ra) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
            } else {
                if (up[0]) ra[0] = o[0].x;
                if (up[1]) ra[1] = o[0].y;
                if (up[2]) ra[2] = o[1].x;
                if (up[3]) ra[3] = o[1].y;
            }
        }
    }
}

template <typename A>
__device__ __forceinline__ A tau_vhs(A rho, A RT, A R, A mu_ref, A T_ref, A omega)
{
    const A T = fdiv(RT, R);
    return fdiv(mu_ref * powa(fdiv(T, T_ref), omega), rho * RT);
}

template <int D, int V, typename T, typename PP>
__device__ __forceinline__ void load_nodes(const PP& P, int k0, T (*x)[D], T* w)
{
    T xx[V * D];
    if constexpr ((V * D * sizeof(T)) % 16 == 0) {
        constexpr int PER = 16 / sizeof(T);
#pragma unroll
        for (int j = 0; j < V * D / PER; ++j) ldv<T, PER>(P.xi + (size_t)k0 * D + j * PER, xx + j * PER);
    } else if constexpr (sizeof(T) == 4 && (V * D) % 2 == 0) {
        // 8-byte pairs (k0 is a multiple of V, so k0 D is even)
#pragma unroll
        for (int j = 0; j < V * D / 2; ++j) ldv<T, 2>(P.xi + (size_t)k0 * D + 2 * j, xx + 2 * j);
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

// FP32 node pair (k, k+1), k even, from the pair layout: X[d] the pair's
// d-th components (one 8- or 16-byte load each), W2 their weights.
template <int D, typename PP>
__device__ __forceinline__ void load_pair(const PP& P, int k, float2 (&X)[D], float2& W2)
{
    const float* p = P.xp + (size_t)k * D;
    if constexpr (D == 2) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        X[0] = make_float2(v.x, v.y);
        X[1] = make_float2(v.z, v.w);
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) X[d] = *reinterpret_cast<const float2*>(p + 2 * d);
    }
    W2 = *reinterpret_cast<const float2*>(reinterpret_cast<const float*>(P.w) + k);
}

// Four FP32 nodes k..k+3, k a multiple of 4, as two pairs from the pair
// layout (16-byte loads): X[p][d], W2[p] for the pair (k + 2p, k + 2p + 1).
template <int D>
__device__ __forceinline__ void load_quad(const float* xp, const float* w, int k, float2 (&X)[2][D],
                                          float2 (&W2)[2])
{
    float xx[4 * D];
    ldvn<float, 4 * D>(xp + (size_t)k * D, xx);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int d = 0; d < D; ++d) X[p][d] = make_float2(xx[(p * D + d) * 2], xx[(p * D + d) * 2 + 1]);
    const float4 wv = *reinterpret_cast<const float4*>(w + k);
    W2[0] = make_float2(wv.x, wv.y);
    W2[1] = make_float2(wv.z, wv.w);
}

// ------------------------------------------------------------------ k_face
template <int D, typename T>
struct FaceP {
    int Nv, Nvp;
    size_t cstride;          // elements per cell in f: NA * Nvp
    T h;
    double hd;
    double R, Pr, omega, mu_ref, T_ref;
    T* FB;                     // [face][array][Nvp]: foot values phi_bar (k_foot) in,
                               // per-node flux (xi . An) phi_ij out (pass B overwrites in place)
    double* __restrict__ AF;   // [face][D+2] area-weighted flux of W
    const double* __restrict__ Win;
    const T* __restrict__ xi;
    const T* __restrict__ w;
    const float* __restrict__ xp;            // FP32 node coordinates by pairs [Nvp/2][D][2]
    const int* __restrict__ order;
    const int* __restrict__ faceL;
    const int* __restrict__ faceR;
    const T* __restrict__ An;
    const T* __restrict__ rL;
    const T* __restrict__ rR;
    const double* __restrict__ bc;
    int* err;
};

template <typename T>
struct FaceSt {
    int kind, L, R;          // kind: 0 interior, 1 wall, 2 far field
    T An[3], rL[3], rR[3];
    double V[3];             // reference velocity of the moment sums
    T Vt[3];                 // the same in the element type
    EqPar<T> eq;             // interface equilibrium / incoming Maxwellian
    T wa, wb;
};

// The face stage in pieces.  One face, nodes [kb, ke) (thread t of NT owns
// nodes k = kb + tV.., kb + tV + NT V.., V = 2 nodes per iteration):
//   face_setup   (one thread) cells, geometry, reference velocity V of the
//                moment sums (mean of the two cells' velocities), and for a
//                boundary face the incoming Maxwellian (unit density at a wall);
//   face_pass_a  interior: raw moments about V of the foot distribution
//                phi_bar (upwind cell by the sign of xi . An), the foot values
//                kept in shared memory when CACHE; boundary: flux moments of
//                the outgoing foot values and of the incoming Maxwellian;
//   face_state   (one thread, from the summed pass-A moments) the interface
//                state: tau (Eq. 3), q_ij (R4), Shakhov parameters, weights
//                tau/(tau+h), h/(tau+h) (Eq. equ28); wall density from zero
//                net mass flux (R8) and the boundary face's A F;
//   face_pass_b  interior: phi_ij = wa phi_bar + wb g_ij per node, its flux
//                (xi . An) phi_ij and the flux moments
//                sum_k w (xi . An) psi phi_ij; boundary: outgoing foot value /
//                incoming Maxwellian.
// k_face runs them all in one block per face.
template <int D, typename T>
__device__ __forceinline__ void face_setup(const FaceP<D, T>& P, int f, FaceSt<T>& S)
{
    constexpr int NW = D + 2;
    S.L = P.faceL[f];
    S.R = P.faceR[f];
    S.kind = S.R >= 0 ? 0 : (int)P.bc[(size_t)(-1 - S.R) * 6];
    for (int d = 0; d < 3; ++d) {
        S.An[d] = d < D ? P.An[(size_t)f * D + d] : T(0);
        S.rL[d] = d < D ? P.rL[(size_t)f * D + d] : T(0);
        S.rR[d] = d < D ? P.rR[(size_t)f * D + d] : T(0);
        T v = T(0);
        if (d < D) {
            v = (T)P.Win[(size_t)S.L * NW + 1 + d] / (T)P.Win[(size_t)S.L * NW];
            if (S.R >= 0) v = T(0.5) * (v + (T)P.Win[(size_t)S.R * NW + 1 + d] / (T)P.Win[(size_t)S.R * NW]);
        }
        S.V[d] = (double)v;
        S.Vt[d] = v;
    }
    if (S.kind != 0) {
        const double* B = P.bc + (size_t)(-1 - S.R) * 6;
        const double Ub[3] = {B[2], B[3], B[4]};
        S.eq = make_eq<D, T>(S.kind == 1 ? 1.0 : B[1], Ub, P.R * B[5], nullptr, P.Pr);
    }
}

// number of pass-A sums per face: NM raw moments (interior) or 2 (D+2) flux
// moments (boundary: outgoing, incoming)
template <int D>
struct FaceNR {
    static constexpr int NM = NMom<D>::v, NW = D + 2;
    static constexpr int v = (NM > 2 * NW) ? NM : 2 * NW;
};

template <int D, typename T, int NT, bool CACHE, int V>
__device__ __forceinline__ void face_pass_a(const FaceP<D, T>& P, const FaceSt<T>& S, T* fc, int kb, int ke,
                                            T* acc, int tid, int f)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    constexpr int NR = FaceNR<D>::v;
    constexpr bool PACK = sizeof(T) == 4 && V == 2;      // FP32 pairs in packed arithmetic
    const bool inter = S.kind == 0;
    T An[D], Vt[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        An[d] = S.An[d];
        Vt[d] = S.Vt[d];
    }
    const int Nvp = P.Nvp;
    const T* fb = P.FB + (size_t)f * NA * Nvp;          // the face's foot values
#pragma unroll
    for (int m = 0; m < NR; ++m) acc[m] = T(0);
    bool packed = false;
    if constexpr (PACK) {
      if (inter) {
        packed = true;
        // FP32 node pairs in packed two-lane arithmetic; per-lane partial sums
        float2 acc2[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc2[m] = bc2(0.0f);
#pragma unroll 2
        for (int k0 = kb + tid * V; k0 < ke; k0 += NT * V) {
            float2 X[D], W2;
            load_pair<D>(P, k0, X, W2);          // pad nodes carry w = 0 and contribute nothing
            float2 F[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) F[a] = __ldcg(reinterpret_cast<const float2*>((const float*)fb + a * Nvp + k0));
            if constexpr (CACHE) {
#pragma unroll
                for (int a = 0; a < NA; ++a) *reinterpret_cast<float2*>((float*)fc + a * Nvp + k0) = F[a];
            }
            float2 xs[D];
#pragma unroll
            for (int d = 0; d < D; ++d) xs[d] = add2(X[d], bc2(-(float)Vt[d]));
            raw_acc2<D>(acc2, xs, mul2(W2, F[0]), NA == 2 ? mul2(W2, F[NA - 1]) : bc2(0.0f));
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = (T)(acc2[m].x + acc2[m].y);
      }
    }
    if (packed) {
    } else if (inter) {
#pragma unroll 2
        for (int k0 = kb + tid * V; k0 < ke; k0 += NT * V) {
            T x[V][D], wv[V];
            load_nodes<D, V>(P, k0, x, wv);      // pad nodes carry w = 0 and contribute nothing
            T fv[NA][V];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                ldv<T, V>(fb + (size_t)a * Nvp + k0, fv[a]);
                if constexpr (CACHE) stv<T, V>(fc + a * Nvp + k0, fv[a]);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T xs[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xs[d] = x[v][d] - Vt[d];
                raw_acc<D>(acc, xs, wv[v] * fv[0][v], NA == 2 ? wv[v] * fv[NA - 1][v] : T(0));
            }
        }
    } else {
#pragma unroll 2
        for (int k0 = kb + tid * V; k0 < ke; k0 += NT * V) {
            T x[V][D], wv[V], sn[V];
            load_nodes<D, V>(P, k0, x, wv);
            T fv[NA][V];
#pragma unroll
            for (int a = 0; a < NA; ++a) ldv<T, V>(fb + (size_t)a * Nvp + k0, fv[a]);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                sn[v] = dot_rn<D>(x[v], An);
                const bool out = sn[v] >= T(0);
                T g0 = fv[0][v], g1 = NA == 2 ? fv[NA - 1][v] : T(0);
                if (!out) eq_eval<D>(S.eq, x[v], g0, g1);
                const T t = wv[v] * sn[v];
                T x2 = T(0);
#pragma unroll
                for (int d = 0; d < D; ++d) x2 += x[v][d] * x[v][d];
                T mm[NW];
                mm[0] = t * g0;
#pragma unroll
                for (int d = 0; d < D; ++d) mm[1 + d] = t * g0 * x[v][d];
                mm[D + 1] = t * T(0.5) * (x2 * g0 + g1);
#pragma unroll
                for (int c = 0; c < NW; ++c) {
                    acc[c] += out ? mm[c] : T(0);
                    acc[NW + c] += out ? T(0) : mm[c];
                }
            }
        }
    }
}

// Interface state from the summed pass-A moments red[]; writes S.eq, S.wa,
// S.wb and, for a boundary face, its area-weighted flux AF[0..D+1].
template <int D, typename T>
__device__ __forceinline__ void face_state(const FaceP<D, T>& P, FaceSt<T>& S, const double* red, double* AF)
{
    constexpr int NW = D + 2;
    if (S.kind == 0) {
        T rho, U[3], RT, qb[3];
        state_from_raw<D, T>(red, S.V, rho, U, RT, qb);
        if (!(rho > T(0)) || !(RT > T(0))) atomicOr(P.err, 1);
        const T tau = tau_vhs<T>(rho, RT, (T)P.R, (T)P.mu_ref, (T)P.T_ref, (T)P.omega);
        const T hh = (T)P.hd;
        T qf[3] = {T(0), T(0), T(0)};
        const T qs = fdiv(tau, tau + hh * (T)P.Pr);
        for (int d = 0; d < D; ++d) qf[d] = qs * qb[d];
        S.eq = make_eq_a<D, T, T>(rho, U, RT, qf, (T)P.Pr);
        S.wa = fdiv(tau, tau + hh);
        S.wb = fdiv(hh, tau + hh);
    } else if (S.kind == 1) {
        const double Sin = -red[NW];          // incoming mass flux of the unit-density wall Maxwellian
        const double rw = Sin > 0.0 ? red[0] / Sin : 0.0;
        for (int m = 0; m < NW; ++m) AF[m] = red[m] + rw * red[NW + m];
        const double* B = P.bc + (size_t)(-1 - S.R) * 6;
        const double Ub[3] = {B[2], B[3], B[4]};
        S.eq = make_eq<D, T>(rw, Ub, P.R * B[5], nullptr, P.Pr);
    } else {
        for (int m = 0; m < NW; ++m) AF[m] = red[m] + red[NW + m];
    }
}

// Pass B over nodes [kb, ke): writes the per-node flux over the face's foot
// values in FB (in place) and, for an interior face, returns the per-thread
// flux-moment partial sums in acc[D+2] (element type).
template <int D, typename T, int NT, bool CACHE, int V>
__device__ __forceinline__ void face_pass_b(const FaceP<D, T>& P, const FaceSt<T>& S, const T* fc, int kb, int ke,
                                            T* acc, int tid, int f)
{
    constexpr int NA = NArr<D>::v, NW = D + 2;
    constexpr bool PACK = sizeof(T) == 4 && V == 2;
    const bool inter = S.kind == 0;
    T An[D];
#pragma unroll
    for (int d = 0; d < D; ++d) An[d] = S.An[d];
    const int Nvp = P.Nvp;
    T* Fo = P.FB + (size_t)f * NA * Nvp;                // foot values in, flux out
#pragma unroll
    for (int m = 0; m < NW; ++m) acc[m] = T(0);
    bool packed = false;
    if constexpr (PACK) {
      if (inter) {
        packed = true;
        const float2 wa = bc2((float)S.wa), wb = bc2((float)S.wb);
        const EqPar<float> eq = *reinterpret_cast<const EqPar<float>*>(&S.eq);
        float2 acc2[NW];
#pragma unroll
        for (int m = 0; m < NW; ++m) acc2[m] = bc2(0.0f);
#pragma unroll 2
        for (int k0 = kb + tid * V; k0 < ke; k0 += NT * V) {
            float2 X[D], W2;
            load_pair<D>(P, k0, X, W2);
            float2 sn = mul2(X[0], bc2(An[0]));
#pragma unroll
            for (int d = 1; d < D; ++d) sn = add2(sn, mul2(X[d], bc2(An[d])));
            float2 F[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a)
                F[a] = CACHE ? *reinterpret_cast<const float2*>((const float*)fc + a * Nvp + k0)
                             : __ldcg(reinterpret_cast<const float2*>((const float*)Fo + a * Nvp + k0));
            float2 gG, gH;
            eq_eval2<D>(eq, X, gG, gH);
            const float2 pG = fma2(wb, gG, mul2(wa, F[0]));
            const float2 pH = NA == 2 ? fma2(wb, gH, mul2(wa, F[NA - 1])) : bc2(0.0f);
            const float2 t = mul2(W2, sn);
            float2 x2 = mul2(X[0], X[0]);
#pragma unroll
            for (int d = 1; d < D; ++d) x2 = fma2(X[d], X[d], x2);
            acc2[0] = fma2(t, pG, acc2[0]);
            const float2 tp = mul2(t, pG);
#pragma unroll
            for (int d = 0; d < D; ++d) acc2[1 + d] = fma2(tp, X[d], acc2[1 + d]);
            acc2[D + 1] = fma2(mul2(t, bc2(0.5f)), fma2(x2, pG, pH), acc2[D + 1]);
            *reinterpret_cast<float2*>((float*)Fo + k0) = mul2(sn, pG);
            if (NA == 2) *reinterpret_cast<float2*>((float*)Fo + (size_t)(NA - 1) * Nvp + k0) = mul2(sn, pH);
        }
#pragma unroll
        for (int m = 0; m < NW; ++m) acc[m] = (T)(acc2[m].x + acc2[m].y);
      }
    }
    if (packed) {
    } else if (inter) {
        const T wa = S.wa, wb = S.wb;
#pragma unroll 2
        for (int k0 = kb + tid * V; k0 < ke; k0 += NT * V) {
            T x[V][D], wv[V], sn[V];
            load_nodes<D, V>(P, k0, x, wv);
#pragma unroll
            for (int v = 0; v < V; ++v) sn[v] = dot_rn<D>(x[v], An);
            T fv[NA][V];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                if constexpr (CACHE) ldv<T, V>(fc + a * Nvp + k0, fv[a]);
                else ldv<T, V>(Fo + (size_t)a * Nvp + k0, fv[a]);
            }
            T o[NA][V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T gG, gH;
                eq_eval<D>(S.eq, x[v], gG, gH);
                const T pG = wa * fv[0][v] + wb * gG;
                const T pH = NA == 2 ? wa * fv[NA - 1][v] + wb * gH : T(0);
                const T t = wv[v] * sn[v];
                T x2 = T(0);
#pragma unroll
                for (int d = 0; d < D; ++d) x2 += x[v][d] * x[v][d];
                acc[0] += t * pG;
#pragma unroll
                for (int d = 0; d < D; ++d) acc[1 + d] += t * pG * x[v][d];
                acc[D + 1] += t * T(0.5) * (x2 * pG + pH);
                o[0][v] = sn[v] * pG;
                if (NA == 2) o[NA - 1][v] = sn[v] * pH;
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) stv<T, V>(Fo + (size_t)a * Nvp + k0, o[a]);
        }
    } else {
#pragma unroll 2
        for (int k0 = kb + tid * V; k0 < ke; k0 += NT * V) {
            T x[V][D], wv[V], sn[V];
            load_nodes<D, V>(P, k0, x, wv);
            T fv[NA][V];
#pragma unroll
            for (int a = 0; a < NA; ++a) ldv<T, V>(Fo + (size_t)a * Nvp + k0, fv[a]);
            T o[NA][V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                sn[v] = dot_rn<D>(x[v], An);
                T g0 = fv[0][v], g1 = NA == 2 ? fv[NA - 1][v] : T(0);
                if (sn[v] < T(0)) eq_eval<D>(S.eq, x[v], g0, g1);
                o[0][v] = sn[v] * g0;
                if (NA == 2) o[NA - 1][v] = sn[v] * g1;
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) stv<T, V>(Fo + (size_t)a * Nvp + k0, o[a]);
        }
    }
}

// One block per face, all nodes: setup, pass A, state, pass B.
template <int D, typename T, int NT, bool CACHE, int VF>
__global__ void __launch_bounds__(NT, NT == 32 ? 32 : ((sizeof(T) == 4) ? (VF == 4 ? 5 : 7) : 4)) k_face(FaceP<D, T> P)
{
    constexpr int NW = D + 2;
    constexpr int NR = FaceNR<D>::v;
    __shared__ FaceSt<T> S;
    __shared__ double sw[(NT / 32) * NR];
    __shared__ double red[NR];
    extern __shared__ __align__(16) unsigned char face_dsm[];
    T* fc = reinterpret_cast<T*>(face_dsm);     // [array][Nvp] foot values (CACHE)

    const int tid = threadIdx.x;
    const int f = P.order[blockIdx.x];
    if (tid == 0) face_setup<D, T>(P, f, S);
    __syncthreads();
    {
        T acc[NR];
        face_pass_a<D, T, NT, CACHE, VF>(P, S, fc, 0, P.Nv, acc, tid, f);
        block_sum_t<NR, NT>(acc, sw, red);
    }
    if (tid == 0) face_state<D, T>(P, S, red, P.AF + (size_t)f * NW);
    __syncthreads();
    T acc[NW];
    face_pass_b<D, T, NT, CACHE, VF>(P, S, fc, 0, P.Nv, acc, tid, f);
    if (S.kind == 0) {
        block_sum_t<NW, NT>(acc, sw, red);
        if (tid < NW) P.AF[(size_t)f * NW + tid] = red[tid];
    }
}

// ---- k_face_staged: the FP32 face kernel for rows beyond the shared-memory
// cache.  Same passes, state and arithmetic as k_face's packed path; the
// face's foot-value row (and, with SXI, the node coordinates and weights,
// which otherwise come by direct loads) reach shared memory by asynchronous
// 1D bulk copies in stages of CH nodes, double-buffered on two mbarriers, so
// that the loads of stage g+1 (and the first stages of pass B, during the
// state computation) overlap the work on stage g.  Offsets and sizes are multiples of 16 bytes by construction (rows
// of Nvp = 32 m nodes, stages of CH = 32 n nodes, the last one cut at Nvp).  Every
// wait is bounded (about a second); a wait that gives up sets bit 4 of the
// error word (AVS_ETIMEOUT at the next blocking call) and the block drains its
// copies, again with a bound, before it leaves.
template <int D, int CH, bool SXI>
struct StageFloats { static constexpr int v = (NArr<D>::v + (SXI ? D + 1 : 0)) * CH; };
constexpr long long kWaitCycles = 2000000000ll;

template <int D, int NT, int CH, bool SXI>
__global__ void __launch_bounds__(NT, NT == 64 ? 13 : 7) k_face_staged(FaceP<D, float> P)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    constexpr int NR = FaceNR<D>::v;
    static_assert(CH % 32 == 0 && CH % (4 * NT) == 0, "stage: whole node quads per thread, 128-byte rows");
    // node loop: with the coordinates loaded directly, quads (two 16-byte
    // pair loads per coordinate block); with them staged, pairs (measured on
    // GB300: 3D 68.1 against 70.4 ms per UGKS step, 2D 9.92 against 10.0)
    constexpr bool QUAD = !SXI;
    __shared__ FaceSt<float> S;
    __shared__ double sw[(NT / 32) * NR];
    __shared__ double red[NR];
    extern __shared__ __align__(128) float stg[];   // two stages of SF floats
    constexpr int SF = StageFloats<D, CH, SXI>::v;
    __shared__ __align__(8) unsigned long long full[2];
    __shared__ int bad, gbad, nissued;           // timeout flag, first stage given up, stages issued

    const int tid = threadIdx.x;
    const int f = P.order[blockIdx.x];
    if (tid == 0) {
        face_setup<D, float>(P, f, S);
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
        bad = 0;
        gbad = 1 << 30;
        nissued = 0;
    }
    __syncthreads();
    if (S.kind != 0) {
        // boundary face: the direct-load passes
        float acc[NR];
        face_pass_a<D, float, NT, false, 2>(P, S, nullptr, 0, P.Nv, acc, tid, f);
        block_sum_t<NR, NT>(acc, sw, red);
        if (tid == 0) face_state<D, float>(P, S, red, P.AF + (size_t)f * NW);
        __syncthreads();
        float accb[NW];
        face_pass_b<D, float, NT, false, 2>(P, S, nullptr, 0, P.Nv, accb, tid, f);
        return;
    }
    const int Nv = P.Nv, Nvp = P.Nvp;
    const int nst = (Nv + CH - 1) / CH;          // stages per pass
    const int ng = 2 * nst;                      // pass A stages, then pass B stages
    float* row = P.FB + (size_t)f * NA * Nvp;
    auto issue = [&](int g) {                    // thread 0
        const int b = g & 1;
        const int k0 = (g < nst ? g : g - nst) * CH;
        const int n = min(CH, Nvp - k0);         // a multiple of 32 nodes
        const unsigned bytes = (unsigned)n * 4u;
        float* dst = stg + b * SF;
        nissued = g + 1;
        mbar_arrive_expect_tx(&full[b], bytes * (unsigned)(NA + (SXI ? D + 1 : 0)));
#pragma unroll
        for (int a = 0; a < NA; ++a) bulk_g2s(dst + a * CH, row + (size_t)a * Nvp + k0, bytes, &full[b]);
        if constexpr (SXI) {
            bulk_g2s(dst + NA * CH, P.xp + (size_t)k0 * D, bytes * D, &full[b]);
            bulk_g2s(dst + (NA + D) * CH, P.w + k0, bytes, &full[b]);
        }
    };
    // node pair (k, k+1) = stage offsets (kk, kk+1): from the stage, or
    // direct loads (the coordinates and weights are shared by all faces)
    auto stage_nodes = [&](const float* st, int k, int kk, float2 (&X)[D], float2& W2) {
        if constexpr (SXI) {
            const float* xv = st + NA * CH + kk * D;      // pair layout, as in P.xp
#pragma unroll
            for (int d = 0; d < D; ++d) X[d] = *reinterpret_cast<const float2*>(xv + 2 * d);
            W2 = *reinterpret_cast<const float2*>(st + (NA + D) * CH + kk);
        } else {
            load_pair<D>(P, k, X, W2);
        }
    };
    auto wait = [&](int g) {
        if (bad) return;                         // a wait gave up: no further waits
        if (!mbar_wait_bounded(&full[g & 1], (unsigned)((g >> 1) & 1), kWaitCycles)) {
            atomicOr(P.err, 4);
            atomicMin(&gbad, g);
            bad = 1;
        }
    };
    if (tid == 0) {
        // after a wait that gave up anywhere, later blocks issue no copies
        if (*(volatile int*)P.err & 4) bad = 2;
        if (!bad) {
            issue(0);
            if (ng > 1) issue(1);
        }
    }
    __syncthreads();
    if (bad) return;
    float Vt[D], An[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        Vt[d] = S.Vt[d];
        An[d] = S.An[d];
    }
    // ---------------- pass A: raw moments of the foot values about V
    float2 acc2[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc2[m] = bc2(0.0f);
    for (int g = 0; g < nst; ++g) {
        wait(g);
        const float* st = stg + (g & 1) * SF;
        const int k0 = g * CH;
        auto bodyA = [&](int kk, const float2 (&X)[D], float2 W2) {
            float2 F[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) F[a] = *reinterpret_cast<const float2*>(st + a * CH + kk);
            float2 xs[D];
#pragma unroll
            for (int d = 0; d < D; ++d) xs[d] = add2(X[d], bc2(-Vt[d]));
            raw_acc2<D>(acc2, xs, mul2(W2, F[0]), NA == 2 ? mul2(W2, F[NA - 1]) : bc2(0.0f));
        };
        if constexpr (QUAD) {
#pragma unroll 1
            for (int kq = tid * 4; kq < CH; kq += NT * 4) {
                if (k0 + kq >= Nv) break;        // the quad's pad nodes carry w = 0
                float2 XQ[2][D], WQ[2];
                load_quad<D>(P.xp, P.w, k0 + kq, XQ, WQ);
                bodyA(kq, XQ[0], WQ[0]);
                bodyA(kq + 2, XQ[1], WQ[1]);
            }
        } else {
#pragma unroll 4
            for (int kk = tid * 2; kk < CH; kk += NT * 2) {
                if (k0 + kk >= Nv) break;
                float2 X[D], W2;
                stage_nodes(st, k0 + kk, kk, X, W2);
                bodyA(kk, X, W2);
            }
        }
        __syncthreads();
        if (tid == 0 && g + 2 < ng && !bad) {
            fence_proxy_async_smem();
            issue(g + 2);
        }
    }
    {
        float acc[NR];
#pragma unroll
        for (int m = 0; m < NR; ++m) acc[m] = m < NM ? acc2[m].x + acc2[m].y : 0.0f;
        block_sum_t<NR, NT>(acc, sw, red);
    }
    if (tid == 0) face_state<D, float>(P, S, red, P.AF + (size_t)f * NW);
    __syncthreads();
    // ---------------- pass B: per-node flux of the interface distribution
    const float2 wa = bc2(S.wa), wb = bc2(S.wb);
    const EqPar<float> eq = S.eq;
    float2 accB[NW];
#pragma unroll
    for (int m = 0; m < NW; ++m) accB[m] = bc2(0.0f);
    for (int g = nst; g < ng; ++g) {
        wait(g);
        const float* st = stg + (g & 1) * SF;
        const int k0 = (g - nst) * CH;
        auto bodyB = [&](int kk, const float2 (&X)[D], float2 W2) {
            const int k = k0 + kk;
            float2 F[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) F[a] = *reinterpret_cast<const float2*>(st + a * CH + kk);
            float2 sn = mul2(X[0], bc2(An[0]));
#pragma unroll
            for (int d = 1; d < D; ++d) sn = add2(sn, mul2(X[d], bc2(An[d])));
            float2 gG, gH;
            eq_eval2<D>(eq, X, gG, gH);
            const float2 pG = fma2(wb, gG, mul2(wa, F[0]));
            const float2 pH = NA == 2 ? fma2(wb, gH, mul2(wa, F[NA - 1])) : bc2(0.0f);
            const float2 t = mul2(W2, sn);
            float2 x2 = mul2(X[0], X[0]);
#pragma unroll
            for (int d = 1; d < D; ++d) x2 = fma2(X[d], X[d], x2);
            accB[0] = fma2(t, pG, accB[0]);
            const float2 tp = mul2(t, pG);
#pragma unroll
            for (int d = 0; d < D; ++d) accB[1 + d] = fma2(tp, X[d], accB[1 + d]);
            accB[D + 1] = fma2(mul2(t, bc2(0.5f)), fma2(x2, pG, pH), accB[D + 1]);
            *reinterpret_cast<float2*>(row + k) = mul2(sn, pG);
            if (NA == 2) *reinterpret_cast<float2*>(row + (size_t)(NA - 1) * Nvp + k) = mul2(sn, pH);
        };
        if constexpr (QUAD) {
#pragma unroll 1
            for (int kq = tid * 4; kq < CH; kq += NT * 4) {
                if (k0 + kq >= Nv) break;        // the quad's pad nodes carry w = 0 and xi = 0
                float2 XQ[2][D], WQ[2];
                load_quad<D>(P.xp, P.w, k0 + kq, XQ, WQ);
                bodyB(kq, XQ[0], WQ[0]);
                bodyB(kq + 2, XQ[1], WQ[1]);
            }
        } else {
#pragma unroll 4
            for (int kk = tid * 2; kk < CH; kk += NT * 2) {
                if (k0 + kk >= Nv) break;
                float2 X[D], W2;
                stage_nodes(st, k0 + kk, kk, X, W2);
                bodyB(kk, X, W2);
            }
        }
        __syncthreads();
        if (tid == 0 && g + 2 < ng && !bad) {
            fence_proxy_async_smem();
            issue(g + 2);
        }
    }
    {
        float acc[NW];
#pragma unroll
        for (int m = 0; m < NW; ++m) acc[m] = accB[m].x + accB[m].y;
        block_sum_t<NW, NT>(acc, sw, red);
        if (tid < NW) P.AF[(size_t)f * NW + tid] = red[tid];
    }
    // a wait that gave up leaves copies in flight: drain them (bounded) before
    // the block's shared memory is released
    if (bad && tid == 0) {
        for (int g = gbad; g < nissued; ++g)
            mbar_wait_bounded(&full[g & 1], (unsigned)((g >> 1) & 1), kWaitCycles);
    }
}

// ------------------------------------------------------------------ k_cell
// Per-cell parameters of the collision update, written by k_cell_state.
template <typename T>
struct CellPar {
    EqPar<T> eq;             // Shakhov(W~, q~) of the cell
    T upd[4];                // 1/dt, 1/tau~, 1/|V|, 1/(1/dt + 1/tau~)
    T Vn[3];                 // U(W~) in the element type: reference of the next raw moments
};

static_assert(sizeof(CellPar<double>) <= AVS_CELLPAR_BYTES, "CellPar buffer size");

template <int D, typename T>
struct CellP {
    int Nc, Nv, Nvp;
    size_t cstride;
    double dt;
    double R, Pr, omega, mu_ref, T_ref;
    const T* __restrict__ fin;
    T* __restrict__ fout;
    const T* __restrict__ F;
    const double* __restrict__ AF;
    const double* __restrict__ Win;
    double* __restrict__ Wout;
    double* mom;             // [cell][NM] raw moments of f about U(W) (read by k_cell_state, rewritten by k_cell)
    CellPar<T>* par;         // [cell]
    const T* __restrict__ xi;
    const T* __restrict__ w;
    const float* __restrict__ xp;            // FP32 node coordinates by pairs [Nvp/2][D][2]
    const int* __restrict__ slot;
    const unsigned char* __restrict__ nslot;
    const double* __restrict__ vol;
    int* err;
};

// Raw moments of the own f^n of cell i about its U(W^n) over nodes [kb, ke):
// per-thread partial sums in acc[NM].
template <int D, typename T, int NT, int VC>
__device__ __forceinline__ void cell_raw_moments(const CellP<D, T>& P, int i, int kb, int ke, T* acc)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    constexpr int V = VC;
    T Vct[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vct[d] = (T)P.Win[(size_t)i * NW + 1 + d] / (T)P.Win[(size_t)i * NW];
    const T* fi = P.fin + (size_t)i * P.cstride;
    if constexpr (sizeof(T) == 4 && V == 4) {
        // FP32: the four nodes as two lane pairs in packed arithmetic (the
        // same pairing and order as cell_update's carried sums)
        float2 acc2[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc2[m] = bc2(0.0f);
        for (int k0 = kb + threadIdx.x * V; k0 < ke; k0 += NT * V) {
            float2 X[2][D], W2[2];
            float f0[V], f1[V];
            load_quad<D>(P.xp, P.w, k0, X, W2);
            ldv<T, V>(fi + k0, f0);
            if (NA == 2) ldv<T, V>(fi + P.Nvp + k0, f1);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float2 xs[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xs[d] = add2(X[p][d], bc2(-Vct[d]));
                raw_acc2<D>(acc2, xs, mul2(W2[p], make_float2(f0[2 * p], f0[2 * p + 1])),
                            NA == 2 ? mul2(W2[p], make_float2(f1[2 * p], f1[2 * p + 1])) : bc2(0.0f));
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = acc2[m].x + acc2[m].y;
    } else {
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = T(0);
        for (int k0 = kb + threadIdx.x * V; k0 < ke; k0 += NT * V) {
            T x[V][D], wv[V], f0[V], f1[V];
            load_nodes<D, V>(P, k0, x, wv);
            ldv<T, V>(fi + k0, f0);
            if (NA == 2) ldv<T, V>(fi + P.Nvp + k0, f1);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T xs[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xs[d] = x[v][d] - Vct[d];
                raw_acc<D>(acc, xs, wv[v] * f0[v], NA == 2 ? wv[v] * f1[v] : T(0));
            }
        }
    }
}

// Raw moments of the own f^n of every cell about its U(W^n) (one block per
// cell); used when the previous step did not leave them (after init, set_f,
// set_W or an adaptation).
template <int D, typename T, int NT, int VC>
__global__ void __launch_bounds__(NT) k_raw_moments(CellP<D, T> P)
{
    constexpr int NM = NMom<D>::v;
    __shared__ double sw[(NT / 32) * NM];
    __shared__ double red[NM];
    const int i = blockIdx.x;
    T acc[NM];
    cell_raw_moments<D, T, NT, VC>(P, i, 0, P.Nv, acc);
    block_sum_t<NM, NT>(acc, sw, red);
    if (threadIdx.x < NM) P.mom[(size_t)i * NM + threadIdx.x] = red[threadIdx.x];
}

// One thread per cell: lagged heat flux q~ from the raw moments of f^n (R3),
// W~ = W - dt/|V| sum_j sgn_j A F_j (R2), tau~ and the Shakhov parameters.
template <int D, typename T>
__global__ void k_cell_state(CellP<D, T> P)
{
    constexpr int NM = NMom<D>::v, NW = D + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.Nc) return;
    const double* Wi = P.Win + (size_t)i * NW;
    double Vc[3] = {0.0, 0.0, 0.0}, m[NM];
    for (int d = 0; d < D; ++d) Vc[d] = (double)((T)Wi[1 + d] / (T)Wi[0]);
    for (int k = 0; k < NM; ++k) m[k] = P.mom[(size_t)i * NM + k];
    T rn, Un[3], RTn, qn[3];
    state_from_raw<D, T>(m, Vc, rn, Un, RTn, qn);
    const int ns = P.nslot[i];
    double Wt[5];
    const double dtv = P.dt / P.vol[i];
    for (int c = 0; c < NW; ++c) {
        double sum = 0.0;
        for (int s = 0; s < ns; ++s) {
            const int sl = P.slot[i * AVS_MAXS + s];
            const double a = P.AF[(size_t)(sl >> 1) * NW + c];
            sum += (sl & 1) ? -a : a;
        }
        Wt[c] = Wi[c] - dtv * sum;
        P.Wout[(size_t)i * NW + c] = Wt[c];
    }
    CellPar<T> cp;
    for (int d = 0; d < 3; ++d) cp.Vn[d] = d < D ? (T)Wt[1 + d] / (T)Wt[0] : T(0);
    double rhod, Ud[3], RTd;
    prim<D>(Wt, rhod, Ud, RTd);
    if (!(rhod > 0.0) || !(RTd > 0.0)) atomicOr(P.err, 1);
    const T rho = (T)rhod, RT = (T)RTd;
    T U[3];
    for (int d = 0; d < 3; ++d) U[d] = (T)Ud[d];
    const T tau = tau_vhs<T>(rho, RT, (T)P.R, (T)P.mu_ref, (T)P.T_ref, (T)P.omega);
    cp.eq = make_eq_a<D, T, T>(rho, U, RT, qn, (T)P.Pr);
    const T idt = (T)(1.0 / P.dt), itau = T(1) / tau;
    cp.upd[0] = idt;
    cp.upd[1] = itau;
    cp.upd[2] = (T)(1.0 / P.vol[i]);
    cp.upd[3] = T(1) / (idt + itau);
    P.par[i] = cp;
}

// Collision update of cell i over nodes [kb, ke): net flux N = sum_j sgn_j F_j
// per node and the update (diagonal of Eq. SGS_phi, R1); pad nodes are written
// as zero.  The raw moments of the new f about U(W~) are summed on the way
// (per-thread partials in acc[NM], same nodes per thread and order as
// cell_raw_moments).  fs, sg: the cell's face indices and signs; cp its
// collision parameters (shared memory).
template <int D, typename T, int NT, int VC>
__device__ __forceinline__ void cell_update(const CellP<D, T>& P, int i, int ns, const int* fs, const T* sg,
                                            const CellPar<T>& cp, int kb, int ke, T* acc)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v;
    constexpr int V = VC;
    const T* fi = P.fin + (size_t)i * P.cstride;
    T* fo = P.fout + (size_t)i * P.cstride;
    const T u0 = cp.upd[0], u1 = cp.upd[1], u2 = cp.upd[2], u3 = cp.upd[3];
    T Vnt[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vnt[d] = cp.Vn[d];
    if constexpr (sizeof(T) == 4 && V == 4) {
        // FP32: the four nodes as two lane pairs in packed arithmetic
        float2 acc2[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc2[m] = bc2(0.0f);
        const float2 U0 = bc2(u0), U1 = bc2(u1), U2n = bc2(-u2), U3 = bc2(u3);
        const EqPar<float> eq = cp.eq;
        for (int k0 = kb + threadIdx.x * V; k0 < ke; k0 += NT * V) {
            float2 XX[2][D], W2[2];
            load_quad<D>(P.xp, P.w, k0, XX, W2);
            float fv[NA][V];
            float2 Nn[NA][2];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                ldv_cg<T, V>(fi + (size_t)a * P.Nvp + k0, fv[a]);
                Nn[a][0] = Nn[a][1] = bc2(0.0f);
            }
#pragma unroll
            for (int s = 0; s < AVS_MAXS; ++s) {
                if (s >= ns) break;
                const float* Fs = P.F + (size_t)fs[s] * NA * P.Nvp + k0;
                const float2 g = bc2(sg[s]);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    float t[V];
                    ldv_cg<T, V>(Fs + (size_t)a * P.Nvp, t);
                    Nn[a][0] = fma2(g, make_float2(t[0], t[1]), Nn[a][0]);
                    Nn[a][1] = fma2(g, make_float2(t[2], t[3]), Nn[a][1]);
                }
            }
            float out[NA][V];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const float2* X = XX[p];
                float2 gG, gH;
                eq_eval2<D>(eq, X, gG, gH);
                const bool r0 = k0 + 2 * p < P.Nv, r1 = k0 + 2 * p + 1 < P.Nv;
                float2 o[NA];
                o[0] = mul2(fma2(Nn[0][p], U2n, fma2(make_float2(fv[0][2 * p], fv[0][2 * p + 1]), U0, mul2(gG, U1))),
                            U3);
                if (NA == 2)
                    o[NA - 1] = mul2(fma2(Nn[NA - 1][p], U2n,
                                          fma2(make_float2(fv[NA - 1][2 * p], fv[NA - 1][2 * p + 1]), U0,
                                               mul2(gH, U1))),
                                     U3);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    out[a][2 * p] = r0 ? o[a].x : 0.0f;
                    out[a][2 * p + 1] = r1 ? o[a].y : 0.0f;
                }
                float2 xs[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xs[d] = add2(X[d], bc2(-Vnt[d]));
                raw_acc2<D>(acc2, xs, mul2(W2[p], make_float2(out[0][2 * p], out[0][2 * p + 1])),
                            NA == 2 ? mul2(W2[p], make_float2(out[NA - 1][2 * p], out[NA - 1][2 * p + 1]))
                                    : bc2(0.0f));
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) stv<T, V>(fo + (size_t)a * P.Nvp + k0, out[a]);
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = acc2[m].x + acc2[m].y;
    } else {
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m] = T(0);
        for (int k0 = kb + threadIdx.x * V; k0 < ke; k0 += NT * V) {
            T x[V][D], wv[V];
            load_nodes<D, V>(P, k0, x, wv);
            T Nn[NA][V], fv[NA][V], out[NA][V];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                ldv_cg<T, V>(fi + (size_t)a * P.Nvp + k0, fv[a]);
#pragma unroll
                for (int v = 0; v < V; ++v) Nn[a][v] = T(0);
            }
#pragma unroll
            for (int s = 0; s < AVS_MAXS; ++s) {
                if (s >= ns) break;
                const T* Fs = P.F + (size_t)fs[s] * NA * P.Nvp + k0;
                const T g = sg[s];
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    T t[V];
                    ldv_cg<T, V>(Fs + (size_t)a * P.Nvp, t);
#pragma unroll
                    for (int v = 0; v < V; ++v) Nn[a][v] += g * t[v];
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                T gG, gH;
                eq_eval<D>(cp.eq, x[v], gG, gH);
                const bool real = k0 + v < P.Nv;
                out[0][v] = real ? (fv[0][v] * u0 + gG * u1 - Nn[0][v] * u2) * u3 : T(0);
                if (NA == 2)
                    out[NA - 1][v] = real ? (fv[NA - 1][v] * u0 + gH * u1 - Nn[NA - 1][v] * u2) * u3 : T(0);
                T xs[D];
#pragma unroll
                for (int d = 0; d < D; ++d) xs[d] = x[v][d] - Vnt[d];
                raw_acc<D>(acc, xs, wv[v] * out[0][v], NA == 2 ? wv[v] * out[NA - 1][v] : T(0));
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) stv<T, V>(fo + (size_t)a * P.Nvp + k0, out[a]);
        }
    }
}

// One block per cell, all nodes; the raw moments of f^{n+1} to P.mom.
template <int D, typename T, int NT, int VC>
__global__ void __launch_bounds__(NT, NT == 32 ? 28 : ((sizeof(T) == 4) ? (VC == 4 ? 7 : 7) : 4)) k_cell(CellP<D, T> P)
{
    constexpr int NM = NMom<D>::v;
    __shared__ int fs[AVS_MAXS];
    __shared__ T sg[AVS_MAXS];
    __shared__ double sw[(NT / 32) * NM];
    __shared__ double red[NM];
    __shared__ CellPar<T> cp;

    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int ns = P.nslot[i];
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        fs[tid] = sl >> 1;
        sg[tid] = (sl & 1) ? T(-1) : T(1);
    }
    if (tid == 32 % NT) cp = P.par[i];
    __syncthreads();
    T acc[NM];
    cell_update<D, T, NT, VC>(P, i, ns, fs, sg, cp, 0, P.Nv, acc);
    block_sum_t<NM, NT>(acc, sw, red);
    if (tid < NM) P.mom[(size_t)i * NM + tid] = red[tid];
}

// ---- k_cell_staged: the FP32 cell kernel with the cell's own f row and its
// faces' flux rows streamed through shared memory in stages of CH nodes by
// asynchronous 1D bulk copies, double-buffered on two mbarriers (the direct
// form waits on its loads: eleven 16-byte rows per four nodes and warp).
// Same arithmetic as cell_update's packed form.  Nodes by pairs, pair kk/2 of
// a stage to thread (kk/2) mod NT, up to the quad boundary Nvq of the real
// nodes (pad nodes written as zero); k_raw_moments_pairs repeats that order,
// so that the carried raw moments equal recomputed ones bit for bit.  nrow:
// rows per stage, NA (1 + largest face count).  Copies start on 128-byte row
// boundaries (Nvp = 32 m) and are multiples of 128 bytes.  Waits are bounded
// as in k_face_staged (bit 4 of the error word).
constexpr int kCellStageMin = 1024;              // nodes above which the 3D cell kernel stages its rows
template <int D, int NT, int CH>
__global__ void __launch_bounds__(NT, 7) k_cell_staged(CellP<D, float> P, int nrow)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v;
    static_assert(CH % 32 == 0 && CH % (2 * NT) == 0, "stage: whole node pairs per thread, 128-byte rows");
    extern __shared__ __align__(128) float stg[];
    __shared__ int fs[AVS_MAXS];
    __shared__ float sg[AVS_MAXS];
    __shared__ double sw[(NT / 32) * NM];
    __shared__ double red[NM];
    __shared__ CellPar<float> cp;
    __shared__ __align__(8) unsigned long long full[2];
    __shared__ int bad, gbad, nissued;           // timeout flag, first stage given up, stages issued

    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    const int ns = P.nslot[i];
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        fs[tid] = sl >> 1;
        sg[tid] = (sl & 1) ? -1.0f : 1.0f;
    }
    if (tid == NT - 1) cp = P.par[i];
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
        bad = 0;
        gbad = 1 << 30;
        nissued = 0;
    }
    __syncthreads();
    const int Nv = P.Nv, Nvp = P.Nvp, Nvq = (Nv + 3) & ~3;
    const int nst = (Nvq + CH - 1) / CH;
    const size_t SF = (size_t)nrow * CH;
    const float* fi = P.fin + (size_t)i * P.cstride;
    float* fo = P.fout + (size_t)i * P.cstride;
    auto issue = [&](int g) {                    // thread 0
        const int b = g & 1;
        const int k0 = g * CH;
        const int n = min(CH, Nvp - k0);         // a multiple of 32 nodes
        const unsigned bytes = (unsigned)n * 4u;
        float* dst = stg + b * SF;
        nissued = g + 1;
        mbar_arrive_expect_tx(&full[b], bytes * (unsigned)(NA * (1 + ns)));
#pragma unroll
        for (int a = 0; a < NA; ++a) bulk_g2s(dst + a * CH, fi + (size_t)a * Nvp + k0, bytes, &full[b]);
        for (int s = 0; s < ns; ++s)
#pragma unroll
            for (int a = 0; a < NA; ++a)
                bulk_g2s(dst + (size_t)(NA * (1 + s) + a) * CH, P.F + ((size_t)fs[s] * NA + a) * Nvp + k0, bytes,
                         &full[b]);
    };
    auto wait = [&](int g) {
        if (bad) return;                         // a wait gave up: no further waits
        if (!mbar_wait_bounded(&full[g & 1], (unsigned)((g >> 1) & 1), kWaitCycles)) {
            atomicOr(P.err, 4);
            atomicMin(&gbad, g);
            bad = 1;
        }
    };
    if (tid == 0) {
        // after a wait that gave up anywhere, later blocks issue no copies
        if (*(volatile int*)P.err & 4) bad = 2;
        if (!bad) {
            issue(0);
            if (nst > 1) issue(1);
        }
    }
    __syncthreads();
    if (bad) return;
    const float2 U0 = bc2(cp.upd[0]), U1 = bc2(cp.upd[1]), U2n = bc2(-cp.upd[2]), U3 = bc2(cp.upd[3]);
    const EqPar<float> eq = cp.eq;
    float Vnt[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vnt[d] = cp.Vn[d];
    float2 acc2[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc2[m] = bc2(0.0f);
    for (int g = 0; g < nst; ++g) {
        wait(g);
        const float* st = stg + (g & 1) * SF;
        const int k0 = g * CH;
        for (int kk = tid * 2; kk < CH; kk += NT * 2) {
            const int k = k0 + kk;
            if (k >= Nvq) break;
            float2 X[D], W2;
            load_pair<D>(P, k, X, W2);
            float2 fv[NA], Nn[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                fv[a] = *reinterpret_cast<const float2*>(st + a * CH + kk);
                Nn[a] = bc2(0.0f);
            }
#pragma unroll
            for (int s = 0; s < AVS_MAXS; ++s) {
                if (s >= ns) break;
                const float2 gs = bc2(sg[s]);
#pragma unroll
                for (int a = 0; a < NA; ++a)
                    Nn[a] = fma2(gs, *reinterpret_cast<const float2*>(st + (NA * (1 + s) + a) * CH + kk), Nn[a]);
            }
            float2 gG, gH;
            eq_eval2<D>(eq, X, gG, gH);
            const bool r0 = k < Nv, r1 = k + 1 < Nv;
            float2 o[NA];
            o[0] = mul2(fma2(Nn[0], U2n, fma2(fv[0], U0, mul2(gG, U1))), U3);
            if (NA == 2) o[NA - 1] = mul2(fma2(Nn[NA - 1], U2n, fma2(fv[NA - 1], U0, mul2(gH, U1))), U3);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                o[a] = make_float2(r0 ? o[a].x : 0.0f, r1 ? o[a].y : 0.0f);
                *reinterpret_cast<float2*>(fo + (size_t)a * Nvp + k) = o[a];
            }
            float2 xs[D];
#pragma unroll
            for (int d = 0; d < D; ++d) xs[d] = add2(X[d], bc2(-Vnt[d]));
            raw_acc2<D>(acc2, xs, mul2(W2, o[0]), NA == 2 ? mul2(W2, o[NA - 1]) : bc2(0.0f));
        }
        __syncthreads();
        if (tid == 0 && g + 2 < nst && !bad) {
            fence_proxy_async_smem();
            issue(g + 2);
        }
    }
    float acc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = acc2[m].x + acc2[m].y;
    block_sum_t<NM, NT>(acc, sw, red);
    if (tid < NM) P.mom[(size_t)i * NM + tid] = red[tid];
    // a wait that gave up leaves copies in flight: drain them (bounded) before
    // the block's shared memory is released
    if (bad && tid == 0) {
        for (int g = gbad; g < nissued; ++g)
            mbar_wait_bounded(&full[g & 1], (unsigned)((g >> 1) & 1), kWaitCycles);
    }
}

// Raw moments of the own FP32 f of every cell about its U(W) in the node
// order of k_cell_staged (pairs kk/2 of each CH-node stage to thread
// (kk/2) mod NT, up to the quad boundary), one block per cell.
template <int D, int NT, int CH>
__global__ void __launch_bounds__(NT) k_raw_moments_pairs(CellP<D, float> P)
{
    constexpr int NA = NArr<D>::v, NM = NMom<D>::v, NW = D + 2;
    __shared__ double sw[(NT / 32) * NM];
    __shared__ double red[NM];
    const int tid = threadIdx.x;
    const int i = blockIdx.x;
    float Vct[D];
#pragma unroll
    for (int d = 0; d < D; ++d) Vct[d] = (float)P.Win[(size_t)i * NW + 1 + d] / (float)P.Win[(size_t)i * NW];
    const int Nv = P.Nv, Nvp = P.Nvp, Nvq = (Nv + 3) & ~3;
    const int nst = (Nvq + CH - 1) / CH;
    const float* fi = P.fin + (size_t)i * P.cstride;
    float2 acc2[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc2[m] = bc2(0.0f);
    for (int g = 0; g < nst; ++g) {
        const int k0 = g * CH;
        for (int kk = tid * 2; kk < CH; kk += NT * 2) {
            const int k = k0 + kk;
            if (k >= Nvq) break;
            float2 X[D], W2;
            load_pair<D>(P, k, X, W2);
            float2 fv[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) fv[a] = *reinterpret_cast<const float2*>(fi + (size_t)a * Nvp + k);
            float2 xs[D];
#pragma unroll
            for (int d = 0; d < D; ++d) xs[d] = add2(X[d], bc2(-Vct[d]));
            raw_acc2<D>(acc2, xs, mul2(W2, fv[0]), NA == 2 ? mul2(W2, fv[NA - 1]) : bc2(0.0f));
        }
    }
    float acc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = acc2[m].x + acc2[m].y;
    block_sum_t<NM, NT>(acc, sw, red);
    if (tid < NM) P.mom[(size_t)i * NM + tid] = red[tid];
}

// k_grad for the FP32 form in packed two-lane arithmetic: four nodes per
// thread as two pairs; the cell's geometry staged once per block in shared
// memory; the gradient and limiter of k_foot_f2, stored as k_grad stores
// them ([cell][array][D][Nvp]).  128-thread blocks, eight per SM.
template <int D, int NS, int NA>
__global__ void __launch_bounds__(128, 8) k_grad_f2(int Nv, int Nvp, int limiter, const float* __restrict__ f,
                                                    float* __restrict__ Gout, CellGeo<float> geo)
{
    constexpr int VG = 4;
    const int i = blockIdx.x;
    const int t = threadIdx.x;
    const int k0 = (blockIdx.y * blockDim.x + t) * VG;
    const int ns = geo.ns[i];
    __shared__ __align__(16) float gs[2][NS][4];      // LSQ weights, face offsets per slot
    __shared__ int gn[NS];                            // neighbour cells (the cell itself where none)
    if (t < NS * 4) {
        const int s = t >> 2, d = t & 3;
        const bool on = s < ns && d < D;
        gs[0][s][d] = on ? geo.cg[(size_t)(i * AVS_MAXS + s) * D + d] : 0.0f;
        gs[1][s][d] = on ? geo.r[(size_t)(i * AVS_MAXS + s) * D + d] : 0.0f;
    } else if (t >= 32 && t < 32 + NS) {
        const int s = t - 32;
        const int n = s < ns ? geo.nbr[i * AVS_MAXS + s] : -1;
        gn[s] = n >= 0 ? n : i;
    }
    __syncthreads();
    if (k0 >= Nv) return;
    const size_t cstride = (size_t)NA * Nvp;
    auto vec = [&](int q, int s, float (&o)[D]) {
        const float4 v = *reinterpret_cast<const float4*>(gs[q][s]);
        o[0] = v.x;
        o[1] = v.y;
        if constexpr (D == 3) o[2] = v.z;
    };
    const float e2 = geo.eps2[i];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const float* fa = f + (size_t)a * Nvp + k0;
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(fa + (size_t)i * cstride));
        const float2 phi[2] = {lo2(c4), hi2(c4)};
        float4 n4[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) n4[s] = __ldg(reinterpret_cast<const float4*>(fa + (size_t)gn[s] * cstride));
        float2 G[D][2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float2 g[D], dd[NS];
#pragma unroll
            for (int d = 0; d < D; ++d) g[d] = bc2(0.0f);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                float cg[D];
                vec(0, s, cg);
                dd[s] = sub2(p ? hi2(n4[s]) : lo2(n4[s]), phi[p]);
#pragma unroll
                for (int d = 0; d < D; ++d) g[d] = fma2(bc2(cg[d]), dd[s], g[d]);
            }
            float2 L = bc2(1.0f);
            if (limiter == 1) {
                float2 d2[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    float rr[D];
                    vec(1, s, rr);
                    d2[s] = mul2(g[0], bc2(rr[0]));
#pragma unroll
                    for (int d = 1; d < D; ++d) d2[s] = fma2(g[d], bc2(rr[d]), d2[s]);
                }
                float dx[NS], dy[NS], ex[NS], ey[NS];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    dx[s] = dd[s].x; dy[s] = dd[s].y;
                    ex[s] = d2[s].x; ey[s] = d2[s].y;
                }
                float2 dmax, dmin, pp, nn;
                ext4<NS>(dx, dmax.x, dmin.x);
                ext4<NS>(dy, dmax.y, dmin.y);
                ext4<NS>(ex, pp.x, nn.x);
                ext4<NS>(ey, pp.y, nn.y);
                // epsilon^2 = (K dx)^3 phi_C^2: scaled to the limited value (R6)
                const float2 e2p = mul2(mul2(bc2(e2), phi[p]), phi[p]);
                const float2 tp = venkat2(dmax, pp, e2p);
                const float2 tn = venkat2(dmin, nn, e2p);
                if (pp.x > 0.0f) L.x = tp.x;
                if (pp.y > 0.0f) L.y = tp.y;
                if (nn.x < 0.0f && tn.x < L.x) L.x = tn.x;
                if (nn.y < 0.0f && tn.y < L.y) L.y = tn.y;
            }
            if (limiter == 0) L = bc2(0.0f);
#pragma unroll
            for (int d = 0; d < D; ++d) G[d][p] = mul2(L, g[d]);
        }
        float* o = Gout + ((size_t)i * NA + a) * D * Nvp + k0;
#pragma unroll
        for (int d = 0; d < D; ++d)
            *reinterpret_cast<float4*>(o + (size_t)d * Nvp) = make_float4(G[d][0].x, G[d][0].y, G[d][1].x, G[d][1].y);
    }
}

// Limited gradients of every array of every cell into c->grad (allocated by the caller).
template <int D, typename T, int NA>
static void grad_t(avs_ctx* c, const void* fin)
{
    const bool f32 = sizeof(T) == 4;
    CellGeo<T> geo;
    geo.nbr = c->nbr;
    geo.cg = f32 ? (const T*)c->cg_f : (const T*)c->cg_d;
    geo.r = f32 ? (const T*)c->r_f : (const T*)c->r_d;
    geo.eps2 = f32 ? (const T*)c->eps2_f : (const T*)c->eps2_d;
    geo.ns = c->nslot;
    constexpr int VG = 4;
    if constexpr (sizeof(T) == 4) {
        const dim3 g2(c->Nc, (c->Nv + 128 * VG - 1) / (128 * VG));
        if (D == 2 && c->max_ns <= 4)
            k_grad_f2<D, 4, NA><<<g2, 128, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (const float*)fin,
                                                          (float*)c->grad, geo);
        else
            k_grad_f2<D, AVS_MAXS, NA><<<g2, 128, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (const float*)fin,
                                                                 (float*)c->grad, geo);
        c->launches += 1;
        return;
    }
    dim3 g(c->Nc, (c->Nv + 256 * VG - 1) / (256 * VG));
    if (D == 2 && c->max_ns <= 4)
        k_grad<D, T, VG, 4, NA><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (const T*)fin, (T*)c->grad, geo);
    else
        k_grad<D, T, VG, AVS_MAXS, NA><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (const T*)fin,
                                                                  (T*)c->grad, geo);
    c->launches += 1;
}

// Foot values of every face (k_foot) and the face stage of a step: per-node
// face flux in c->flux, area-weighted face flux of W in c->AFf (shared by
// the explicit and the implicit step).
template <int D, typename T>
static cudaError_t face_stage_t(avs_ctx* c, const void* fin, const double* Win, double dt)
{
    const bool f32 = sizeof(T) == 4;
    const int NA = NArr<D>::v;
    const size_t rows = (size_t)std::max(c->fcap, c->Nvp);   // sized for the f capacity: no reallocation
    {
        // foot values, then (in place) the face flux; afterwards one f-sized
        // array for the implicit step's increment
        const size_t need = (size_t)std::max(c->Nf, c->Nc) * NA * rows * sizeof(T);
        if (c->flux_bytes < need) {
            if (c->flux) cudaFree(c->flux);
            c->flux = nullptr;
            c->flux_bytes = 0;
            cudaError_t e = cudaMalloc(&c->flux, need);
            if (e != cudaSuccess) return e;
            c->flux_bytes = need;
        }
    }
    const T* xi = f32 ? (const T*)c->xi_f : (const T*)c->xi_d;
    const T* w = f32 ? (const T*)c->w_f : (const T*)c->w_d;
    const T* An = f32 ? (const T*)c->An_f : (const T*)c->An_d;
    const double hd = 0.5 * dt;
    {
        CellGeo<T> geo;
        geo.nbr = c->nbr;
        geo.cg = f32 ? (const T*)c->cg_f : (const T*)c->cg_d;
        geo.r = f32 ? (const T*)c->r_f : (const T*)c->r_d;
        geo.eps2 = f32 ? (const T*)c->eps2_f : (const T*)c->eps2_d;
        geo.ns = c->nslot;
        constexpr int VG = 4;
        const dim3 g(c->Nc, (c->Nv + 256 * VG - 1) / (256 * VG));
        if constexpr (sizeof(T) == 4) {
            // 128-thread blocks, eight per SM (measured on GB300: 1-2 % faster
            // per UGKS step than 256-thread blocks, four per SM)
            const dim3 g2(c->Nc, (c->Nv + 128 * VG - 1) / (128 * VG));
            if (D == 2 && c->max_ns <= 4)
                k_foot_f2<D, 4, NArr<D>::v><<<g2, 128, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (float)hd,
                                                                      (const float*)fin, (float*)c->flux, geo,
                                                                      c->slot, An, c->xi_p);
            else
                k_foot_f2<D, AVS_MAXS, NArr<D>::v><<<g2, 128, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter,
                                                                             (float)hd, (const float*)fin,
                                                                             (float*)c->flux, geo, c->slot, An,
                                                                             c->xi_p);
        } else if (D == 2 && c->max_ns <= 4) {
            k_foot<D, T, VG, 4, NArr<D>::v><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (T)hd,
                                                                      (const T*)fin, (T*)c->flux, geo, c->slot, An, xi);
        } else {
            k_foot<D, T, VG, AVS_MAXS, NArr<D>::v><<<g, 256, 0, c->stream>>>(c->Nv, c->Nvp, c->cfg.limiter, (T)hd,
                                                                             (const T*)fin, (T*)c->flux, geo, c->slot,
                                                                             An, xi);
        }
        c->launches += 1;
    }
    FaceP<D, T> P;
    P.Nv = c->Nv;
    P.Nvp = c->Nvp;
    P.cstride = (size_t)NA * c->Nvp;
    P.hd = hd;
    P.h = (T)P.hd;
    P.R = c->cfg.R;
    P.Pr = c->cfg.Pr;
    P.omega = c->cfg.omega;
    P.mu_ref = c->mu_ref;
    P.T_ref = c->cfg.T_ref;
    P.FB = (T*)c->flux;
    P.AF = c->AFf;
    P.Win = Win;
    P.xi = xi;
    P.w = w;
    P.xp = c->xi_p;
    P.order = c->forder;
    P.faceL = c->faceL;
    P.faceR = c->faceR;
    P.An = An;
    P.rL = f32 ? (const T*)c->rL_f : (const T*)c->rL_d;
    P.rR = f32 ? (const T*)c->rR_f : (const T*)c->rR_d;
    P.bc = c->bc;
    P.err = c->dev_err;
    constexpr int NT = 128;
    // foot values of pass A kept in shared memory for pass B when they fit in
    // the default dynamic allowance (48 KB); otherwise pass B re-reads the
    // face's row
    const size_t cache_bytes = (size_t)NA * c->Nvp * sizeof(T);
    // two nodes per thread per iteration (8-byte FP32 / 16-byte FP64 vectors):
    // fewer registers and more resident warps than 16-byte FP32 vectors, which
    // the latency-bound face passes prefer; the node loops are unrolled twice
    // so that two iterations' loads are in flight together
    constexpr int VF = 2;
    // small velocity meshes (the Sec. 3.5 spaces): one warp per face, so that
    // threads are not left idle and the block's serial state section holds no
    // other warp; the foot cache then stays small enough for 28+ blocks per SM.
    // Above 256 nodes only with faces enough to fill every SM with such
    // blocks (on fewer faces, 128-thread blocks keep more nodes in flight).
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (cache_bytes <= AVS_SMALL_ROW_BYTES && (c->Nv <= 256 || c->Nf >= 32 * c->nsm)) {
            k_face<D, T, 32, true, VF><<<c->Nf, 32, cache_bytes, c->stream>>>(P);
            done = true;
        }
    }
    // the default allowance covers static and dynamic shared memory together:
    // the block's own arrays (state, reductions: under 2 KB) come first
    constexpr size_t kStaticFace = 2048;
    static_assert(sizeof(FaceSt<T>) + (NT / 32 + 1) * FaceNR<D>::v * sizeof(double) <= kStaticFace,
                  "static shared memory of the face block");
    if (done) {
    } else if (cache_bytes + kStaticFace <= 48 * 1024) {
        k_face<D, T, NT, true, VF><<<c->Nf, NT, cache_bytes, c->stream>>>(P);
    } else if constexpr (sizeof(T) == 4) {
        // rows beyond the cache: bulk-copy stages in shared memory (rows of
        // Nvp = 32 m FP32 values keep every copy 16-byte aligned)
        // measured on GB300 (2D wedge, 12k nodes; 3D sphere, 21k nodes):
        // 2D: stages of 1024 nodes with the node coordinates and weights;
        // 3D: stages of 2048 nodes, coordinates and weights loaded directly
        constexpr int CH = D == 2 ? 1024 : 2048;
        constexpr bool SXI = D == 2;
        constexpr int NTs = D == 2 ? NT : 64;    // 3D: 64-thread face blocks, 13 per SM
        constexpr size_t smem = 2 * sizeof(float) * StageFloats<D, CH, SXI>::v;
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(k_face_staged<D, NTs, CH, SXI>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_face_staged<D, NTs, CH, SXI><<<c->Nf, NTs, smem, c->stream>>>(P);
    } else {
        k_face<D, T, NT, false, VF><<<c->Nf, NT, 0, c->stream>>>(P);
    }
    c->launches += 1;

    return cudaGetLastError();
}

template <int D, typename T>
static cudaError_t launch_step_t(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout,
                                 double dt)
{
    const bool f32 = sizeof(T) == 4;
    const int NA = NArr<D>::v;
    cudaError_t e = face_stage_t<D, T>(c, fin, Win, dt);
    if (e != cudaSuccess) return e;
    const T* xi = f32 ? (const T*)c->xi_f : (const T*)c->xi_d;
    const T* w = f32 ? (const T*)c->w_f : (const T*)c->w_d;
    constexpr int NT = 128;
    CellP<D, T> Q;
    Q.Nc = c->Nc;
    Q.Nv = c->Nv;
    Q.Nvp = c->Nvp;
    Q.cstride = (size_t)NA * c->Nvp;
    Q.dt = dt;
    Q.R = c->cfg.R;
    Q.Pr = c->cfg.Pr;
    Q.omega = c->cfg.omega;
    Q.mu_ref = c->mu_ref;
    Q.T_ref = c->cfg.T_ref;
    Q.fin = (const T*)fin;
    Q.fout = (T*)fout;
    Q.F = (const T*)c->flux;
    Q.AF = c->AFf;
    Q.Win = Win;
    Q.Wout = Wout;
    Q.mom = c->cmom;
    Q.par = (CellPar<T>*)c->cpar;
    Q.xi = xi;
    Q.w = w;
    Q.xp = c->xi_p;
    Q.slot = c->slot;
    Q.nslot = c->nslot;
    Q.vol = c->vol;
    Q.err = c->dev_err;
    // 16-byte vectors (4 FP32 / 2 FP64 nodes per thread) in the cell kernel: it
    // streams f and the face fluxes, and more bytes in flight per warp beat the
    // extra warps of narrower vectors; k_raw_moments uses the same node mapping
    // so that its sums equal the carried ones bit for bit
    constexpr int VC = VW<T>::v;
    // one warp per cell wherever the cells fill every SM with such blocks (and
    // on small velocity meshes): the cell kernel streams its rows, so a warp
    // per cell keeps as many loads in flight and ends with a warp-only
    // reduction; the raw-moment kernel takes the same node mapping (the sums
    // stay the carried ones bit for bit; an adaptation drops them)
    auto cell_stage = [&](auto ntc) {
        constexpr int NTc = decltype(ntc)::value;
        if (!c->mom_valid) {
            k_raw_moments<D, T, NTc, VC><<<c->Nc, NTc, 0, c->stream>>>(Q);
            c->launches += 1;
        }
        k_cell_state<D, T><<<(c->Nc + 127) / 128, 128, 0, c->stream>>>(Q);
        k_cell<D, T, NTc, VC><<<c->Nc, NTc, 0, c->stream>>>(Q);
        c->launches += 2;
    };
    if constexpr (sizeof(T) == 4) {
        if (D == 3 && c->Nv > kCellStageMin) {
            // 3D rows beyond a thousand nodes: the staged cell kernel and the
            // raw-moment kernel of its node order (measured on GB300: 1 %
            // faster on the 21.8k-node sphere; slower in 2D, where the two
            // arrays and four faces take 40 KB of shared memory per block)
            constexpr int NTs = 128, CHs = 512;
            const int nrow = NA * (1 + c->max_ns);
            const size_t smem = 2 * sizeof(float) * (size_t)nrow * CHs;
            if (smem > 48 * 1024) {
                const cudaError_t e = cudaFuncSetAttribute(k_cell_staged<D, NTs, CHs>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
            if (!c->mom_valid) {
                k_raw_moments_pairs<D, NTs, CHs><<<c->Nc, NTs, 0, c->stream>>>(Q);
                c->launches += 1;
            }
            k_cell_state<D, T><<<(c->Nc + 127) / 128, 128, 0, c->stream>>>(Q);
            k_cell_staged<D, NTs, CHs><<<c->Nc, NTs, smem, c->stream>>>(Q, nrow);
            c->launches += 2;
        } else if (c->Nv <= 256 || c->Nc >= 28 * c->nsm) {
            cell_stage(std::integral_constant<int, 32>{});
        } else {
            cell_stage(std::integral_constant<int, NT>{});
        }
    } else {
        cell_stage(std::integral_constant<int, NT>{});
    }
    c->mom_valid = 1;          // the raw moments of fout about U(Wout) are in cmom
    return cudaGetLastError();
}

// ================================================================== implicit step
// IUGKS (Sec. 2.3.1): after the face stage, the macroscopic Eq. (SGS_w) for
// dW = W~ - W^n and the microscopic Eq. (SGS_phi) for dphi are solved by
// symmetric Gauss-Seidel sweeps over a greedy cell colouring: the cells of one
// colour share no face, so a colour is updated in parallel with the values of
// the other colours as they stand, which is the sequential sweep in the order
// "colour 0, colour 1, ..." (forward) and back (backward).

// Euler flux of a conserved state W through the unit normal n (monatomic gas).
template <int D, typename A>
__device__ __forceinline__ void euler_flux_n(const A* W, const A* n, A* G)
{
    const A rho = W[0];
    A m2 = A(0), un = A(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        m2 += W[1 + d] * W[1 + d];
        un += (W[1 + d] / rho) * n[d];
    }
    const A p = rho * ((W[D + 1] - A(0.5) * m2 / rho) / (A(1.5) * rho));
    G[0] = rho * un;
#pragma unroll
    for (int d = 0; d < D; ++d) G[1 + d] = W[1 + d] * un + p * n[d];
    G[D + 1] = (W[D + 1] + p) * un;
}

// Interior face slot of a cell, in sweep order: the slot's outward unit normal
// n, -A/2, A r/2 (r the face's spectral radius) and the Euler flux of the
// neighbour's W^n through n, so that a sweep only evaluates G(W~_j).
template <typename A>
struct ImpSlot {
    A n[3];
    A nhA;
    A hr;
    A Gn[5];
    int j;
};
static_assert(sizeof(ImpSlot<double>) <= AVS_IMPSLOT_BYTES, "slot record");

template <typename A>
struct ImpP {
    int Nc;
    double dt, R, mu_ref, T_ref, omega;
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
    double* Wt;              // W~ [cell][NW] (the output W)
    A* dWa;                  // dW [cell][NW]
    A* Wta;                  // W~ rounded to A [cell][NW]; aliases Wt when A is double
    A* rhs;                  // [q][NW]  -sum sgn A F
    A* dg;                   // [q]      V/dt + 1/2 sum A r
    ImpSlot<A>* co;          // [q][MAXS] interior slots first
    unsigned char* nint;     // [q] interior slots
    const int* clist;        // cells by colour (q -> cell)
    int* err;
};

// Per cell, in sweep order q: diagonal V/dt + 1/2 sum A r over every slot,
// explicit residual -sum sgn A F, and the interior slot records.  r from the
// face's own orientation (L, R, n_LR), so both cells of a face use one value.
template <int D, typename A>
__global__ void k_imp_setup(ImpP<A> P)
{
    constexpr int NW = D + 2;
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
        // spectral radius |U.n| + a + 2 mu / (rho dl) from the mean primitive state
        double rl, Ul[3], RTl, rr, Ur[3], RTr;
        prim<D>(P.Wn + (size_t)L * NW, rl, Ul, RTl);
        prim<D>(P.Wn + (size_t)(R >= 0 ? R : L) * NW, rr, Ur, RTr);
        const double rho = 0.5 * (rl + rr), RT = 0.5 * (RTl + RTr);
        double un = 0.0;
        for (int d = 0; d < D; ++d) un += 0.5 * (Ul[d] + Ur[d]) * n[d];
        const double mu = P.mu_ref * pow(RT / P.R / P.T_ref, P.omega);
        const double r = Aa * (fabs(un) + sqrt(5.0 / 3.0 * RT) + 2.0 * mu / (rho * dl));
        dg += 0.5 * r;
        const int j = (sl & 1) ? L : R;
        if (j >= 0) {
            ImpSlot<A> sc;
            for (int d = 0; d < 3; ++d) sc.n[d] = d < D ? (A)(sgn * An[d] / Aa) : A(0);
            sc.nhA = (A)(-0.5 * Aa);
            sc.hr = (A)(0.5 * r);
            A Wj[NW];
            for (int c = 0; c < NW; ++c) Wj[c] = (A)P.Wn[(size_t)j * NW + c];
            euler_flux_n<D, A>(Wj, sc.n, sc.Gn);
            for (int c = NW; c < 5; ++c) sc.Gn[c] = A(0);
            sc.j = j;
            P.co[(size_t)q * AVS_MAXS + nint++] = sc;
        }
    }
    P.dg[q] = (A)dg;
    P.nint[q] = (unsigned char)nint;
}

// Self-test of the bounded grid barrier: `rounds` barriers, the last one
// waiting for `short_by` arrivals more than the grid has (none when 0), each
// passed barrier counted once per block in *passed.
__global__ void k_grid_barrier_check(unsigned* bar, int rounds, int short_by, int* err, int* passed)
{
    unsigned gen = 0;
    for (int r = 0; r < rounds; ++r) {
        const unsigned target = ++gen * gridDim.x + (r == rounds - 1 ? (unsigned)short_by : 0u);
        if (!grid_sync_bounded(bar, target, err)) return;
        if (threadIdx.x == 0) atomicAdd(passed, 1);
    }
}

cudaError_t launch_grid_barrier_check(avs_ctx* c, int blocks, int rounds, int short_by, int* passed_dev)
{
    cudaError_t e = cudaMemsetAsync(c->imp_bar, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    unsigned* bar = c->imp_bar;
    int* err = c->dev_err;
    void* args[] = {&bar, &rounds, &short_by, &err, &passed_dev};
    e = cudaLaunchCooperativeKernel((const void*)k_grid_barrier_check, dim3(blocks), dim3(128), args, 0, c->stream);
    if (e == cudaSuccess) c->launches += 1;
    return e;
}

// Self-test of the bounded mbarrier wait of the staged kernels: with `arrive`
// one 128-byte bulk copy completes the barrier and the copied bytes are
// compared with the source; without, no arrival ever comes and every thread's
// wait gives up after kWaitCycles, setting bit 4 of the error word.
__global__ void k_stage_wait_check(const float* __restrict__ src, int arrive, int* err, int* completed)
{
    __shared__ __align__(128) float buf[32];
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && arrive) {
        mbar_arrive_expect_tx(&bar, 128u);
        bulk_g2s(buf, src, 128u, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0u, kWaitCycles);
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(err, 4);
            // a copy that was issued may still land: wait for it (bounded)
            if (arrive) mbar_wait_bounded(&bar, 0u, kWaitCycles);
        }
        return;
    }
    if (threadIdx.x == 0) {
        int same = 1;
        for (int j = 0; j < 32; ++j) same &= buf[j] == src[j];
        *completed = same;
    }
}

cudaError_t launch_stage_wait_check(avs_ctx* c, const float* src, bool arrive, int* completed_dev)
{
    k_stage_wait_check<<<1, 32, 0, c->stream>>>(src, arrive ? 1 : 0, c->dev_err, completed_dev);
    c->launches += 1;
    return cudaGetLastError();
}

// One cell of a macroscopic sweep: dW_i = (Res_i(W~) + 1/2 sum A r dW_j) / diag_i,
// Res_i = -sum sgn A F - 1/2 sum A (G(W~_j) - G(W^n_j)) over the interior faces.
// Arithmetic in A (FP32 in the mixed form, where dW is a small correction of
// the FP64 W^n); W~ = W^n + dW in FP64.  The neighbours' values are read past
// L1: other blocks wrote them before the last grid barrier.
template <int D, typename A>
__device__ __forceinline__ void imp_macro_cell(const ImpP<A>& P, int q)
{
    constexpr int NW = D + 2;
    const int i = P.clist[q];
    const int n = P.nint[q];
    A rhs[NW];
#pragma unroll
    for (int c = 0; c < NW; ++c) rhs[c] = P.rhs[(size_t)q * NW + c];
    for (int s = 0; s < n; ++s) {
        const ImpSlot<A> sc = P.co[(size_t)q * AVS_MAXS + s];
        A Wj[NW], dWj[NW], G[NW];
#pragma unroll
        for (int c = 0; c < NW; ++c) {
            Wj[c] = __ldcg(P.Wta + (size_t)sc.j * NW + c);
            dWj[c] = __ldcg(P.dWa + (size_t)sc.j * NW + c);
        }
        euler_flux_n<D, A>(Wj, sc.n, G);
#pragma unroll
        for (int c = 0; c < NW; ++c) rhs[c] += sc.nhA * (G[c] - sc.Gn[c]) + sc.hr * dWj[c];
    }
    const A dg = P.dg[q];
#pragma unroll
    for (int c = 0; c < NW; ++c) {
        const A d = rhs[c] / dg;
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

// The whole macroscopic solve in one cooperative launch: k_macro symmetric
// Gauss-Seidel iterations, each colour a grid-stride pass, a grid barrier
// between passes.  A colour that follows itself (the turn of a symmetric
// sweep) is skipped: its neighbours have not changed, so the pass would
// rewrite the same values.
template <int D, typename A, int NT>
__global__ void __launch_bounds__(NT) k_imp_macro(ImpP<A> P, int k_macro, int ncolor, const int* __restrict__ cstart,
                                                  unsigned* bar)
{
    const unsigned nb = gridDim.x;
    unsigned gen = 0;
    int prev = -1;
    for (int it = 0; it < k_macro; ++it)
        for (int dir = 0; dir < 2; ++dir)
            for (int qq = 0; qq < ncolor; ++qq) {
                const int col = dir == 0 ? qq : ncolor - 1 - qq;
                if (col == prev) continue;
                if (prev >= 0 && !grid_sync_bounded(bar, ++gen * nb, P.err)) return;
                prev = col;
                const int c1 = cstart[col + 1];
                for (int q = cstart[col] + blockIdx.x * NT + threadIdx.x; q < c1; q += nb * NT)
                    imp_macro_cell<D, A>(P, q);
            }
}

// Per cell: Shakhov state of W~ with the lagged heat flux of f^n (R3);
// upd[0] = V/dt + V/tau~, upd[1] = tau~, upd[2] = V.
template <int D, typename T>
__global__ void k_imp_state(CellP<D, T> P, const double* Wt)
{
    constexpr int NM = NMom<D>::v, NW = D + 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.Nc) return;
    const double* Wi = P.Win + (size_t)i * NW;
    double Vc[3] = {0.0, 0.0, 0.0}, m[NM];
    for (int d = 0; d < D; ++d) Vc[d] = (double)((T)Wi[1 + d] / (T)Wi[0]);
    for (int k = 0; k < NM; ++k) m[k] = P.mom[(size_t)i * NM + k];
    T rn, Un[3], RTn, qn[3];
    state_from_raw<D, T>(m, Vc, rn, Un, RTn, qn);
    double rhod, Ud[3], RTd;
    prim<D>(Wt + (size_t)i * NW, rhod, Ud, RTd);
    if (!(rhod > 0.0) || !(RTd > 0.0)) atomicOr(P.err, 1);
    const T rho = (T)rhod, RT = (T)RTd;
    T U[3];
    for (int d = 0; d < 3; ++d) U[d] = (T)Ud[d];
    CellPar<T> cp;
    const T tau = tau_vhs<T>(rho, RT, (T)P.R, (T)P.mu_ref, (T)P.T_ref, (T)P.omega);
    cp.eq = make_eq_a<D, T, T>(rho, U, RT, qn, (T)P.Pr);
    const T V = (T)P.vol[i];
    cp.upd[0] = V / (T)P.dt + V / tau;
    cp.upd[1] = tau;
    cp.upd[2] = V;
    cp.upd[3] = T(0);
    for (int d = 0; d < 3; ++d) cp.Vn[d] = T(0);
    P.par[i] = cp;
}

// Per cell and node: microscopic residual Res = V (g~ - phi^n) / tau~ - N,
// N the net flux of the cell's faces (written over the f^{n+1} buffer).  V
// consecutive nodes per thread as in k_cell; pad nodes get Res = 0.
template <int D, typename T, int NT, int V>
__global__ void __launch_bounds__(NT) k_imp_res(CellP<D, T> P)
{
    constexpr int NA = NArr<D>::v;
    __shared__ int fs[AVS_MAXS];
    __shared__ T sg[AVS_MAXS];
    __shared__ CellPar<T> cp;
    const int i = blockIdx.x, tid = threadIdx.x;
    const int ns = P.nslot[i];
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        fs[tid] = sl >> 1;
        sg[tid] = (sl & 1) ? T(-1) : T(1);
    }
    if (tid == 32 % NT) cp = P.par[i];
    __syncthreads();
    const T* fi = P.fin + (size_t)i * P.cstride;
    T* ro = P.fout + (size_t)i * P.cstride;
    const T Vc = cp.upd[2], tau = cp.upd[1];
    for (int k0 = tid * V; k0 < P.Nv; k0 += NT * V) {
        T x[V][D], wv[V];
        load_nodes<D, V>(P, k0, x, wv);
        T Nn[NA][V], fv[NA][V];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            ldv_cg<T, V>(fi + (size_t)a * P.Nvp + k0, fv[a]);
#pragma unroll
            for (int v = 0; v < V; ++v) Nn[a][v] = T(0);
        }
#pragma unroll
        for (int s = 0; s < AVS_MAXS; ++s) {
            if (s >= ns) break;
            const T* Fs = P.F + (size_t)fs[s] * NA * P.Nvp + k0;
            const T g = sg[s];
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                T t[V];
                ldv_cg<T, V>(Fs + (size_t)a * P.Nvp, t);
#pragma unroll
                for (int v = 0; v < V; ++v) Nn[a][v] += g * t[v];
            }
        }
        T out[NA][V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            T gG, gH;
            eq_eval<D>(cp.eq, x[v], gG, gH);
            const bool real = k0 + v < P.Nv;
            out[0][v] = real ? Vc * (gG - fv[0][v]) / tau - Nn[0][v] : T(0);
            if (NA == 2) out[NA - 1][v] = real ? Vc * (gH - fv[NA - 1][v]) / tau - Nn[NA - 1][v] : T(0);
        }
#pragma unroll
        for (int a = 0; a < NA; ++a) stv<T, V>(ro + (size_t)a * P.Nvp + k0, out[a]);
    }
}

// One colour of a microscopic sweep: dphi_i = (Res_i - sum_{xi.n<0} (xi.n) dphi_j)
// / (V/dt + V/tau~ + sum_{xi.n>=0} xi.n), every node and array.  V consecutive
// nodes per thread (16-byte vectors); a neighbour's row is read only where one
// of the thread's nodes flows in from it.  Pad nodes get dphi = 0.
template <int D, typename T, int NT, int V>
__global__ void __launch_bounds__(NT) k_imp_micro(CellP<D, T> P, const T* __restrict__ res, T* dphi,
                                                  const T* __restrict__ An, const int* __restrict__ faceL,
                                                  const int* __restrict__ faceR, const int* __restrict__ clist, int c0)
{
    constexpr int NA = NArr<D>::v;
    __shared__ T sA[AVS_MAXS][D];
    __shared__ int snb[AVS_MAXS];
    const int i = clist[c0 + blockIdx.x];
    const int ns = P.nslot[i];
    const int tid = threadIdx.x;
    if (tid < ns) {
        const int sl = P.slot[i * AVS_MAXS + tid];
        const int f = sl >> 1;
#pragma unroll
        for (int d = 0; d < D; ++d) sA[tid][d] = (sl & 1) ? -An[(size_t)f * D + d] : An[(size_t)f * D + d];
        snb[tid] = (sl & 1) ? faceL[f] : faceR[f];
    }
    __syncthreads();
    const int k0 = (blockIdx.y * NT + tid) * V;
    if (k0 >= P.Nv) return;
    const T u0 = P.par[i].upd[0];
    T x[V][D], wv[V];
    load_nodes<D, V>(P, k0, x, wv);
    T sn[AVS_MAXS][V], dg[V];
#pragma unroll
    for (int v = 0; v < V; ++v) dg[v] = T(0);
#pragma unroll
    for (int s = 0; s < AVS_MAXS; ++s) {
        if (s >= ns) break;
        T a[D];
#pragma unroll
        for (int d = 0; d < D; ++d) a[d] = sA[s][d];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            sn[s][v] = dot_rn<D>(x[v], a);
            if (sn[s][v] >= T(0)) dg[v] += sn[s][v];
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) dg[v] = u0 + dg[v];
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        T acc[V];
        ldv_cg<T, V>(res + ((size_t)i * NA + a) * P.Nvp + k0, acc);
#pragma unroll
        for (int s = 0; s < AVS_MAXS; ++s) {
            if (s >= ns) break;
            const int j = snb[s];
            bool in = false;
#pragma unroll
            for (int v = 0; v < V; ++v) in |= sn[s][v] < T(0);
            if (j < 0 || !in) continue;
            T t[V];
            ldv_cg<T, V>(dphi + ((size_t)j * NA + a) * P.Nvp + k0, t);
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (sn[s][v] < T(0)) acc[v] -= sn[s][v] * t[v];
        }
        T o[V];
#pragma unroll
        for (int v = 0; v < V; ++v) o[v] = k0 + v < P.Nv ? acc[v] / dg[v] : T(0);
        stv<T, V>(dphi + ((size_t)i * NA + a) * P.Nvp + k0, o);
    }
}

// f^{n+1} = f^n + dphi (pad nodes zero)
template <typename T>
__global__ void k_imp_finish(int Nrows, int Nv, int Nvp, const T* __restrict__ fin, const T* __restrict__ dphi,
                             T* fout)
{
    const int r = blockIdx.x;
    for (int k = blockIdx.y * blockDim.x + threadIdx.x; k < Nvp; k += gridDim.y * blockDim.x)
        fout[(size_t)r * Nvp + k] = k < Nv ? fin[(size_t)r * Nvp + k] + dphi[(size_t)r * Nvp + k] : T(0);
    (void)Nrows;
}

template <int D, typename T>
static cudaError_t launch_step_implicit_t(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout,
                                          double dt, int k_macro, int k_micro)
{
    const bool f32 = sizeof(T) == 4;
    const int NA = NArr<D>::v, NW = D + 2;
    cudaError_t e = face_stage_t<D, T>(c, fin, Win, dt);
    if (e != cudaSuccess) return e;
    using A = T;     // macroscopic sweep arithmetic: FP32 in the mixed form, FP64 in the FP64 form
    ImpP<A> I;
    I.Nc = c->Nc;
    I.dt = dt;
    I.R = c->cfg.R;
    I.mu_ref = c->mu_ref;
    I.T_ref = c->cfg.T_ref;
    I.omega = c->cfg.omega;
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
    I.co = (ImpSlot<A>*)c->imp_co;
    I.nint = c->imp_nint;
    I.clist = c->clist;
    I.err = c->dev_err;
    const int cb = (c->Nc + 127) / 128;
    k_imp_setup<D, A><<<cb, 128, 0, c->stream>>>(I);
    c->launches += 1;
    const int nc = c->ncolor;
    if (k_macro > 0) {
        // one cooperative launch: every block resident, so the bounded grid
        // barriers between colour passes can complete
        constexpr int NTM = 128;
        int maxcol = 0;
        for (int k = 0; k < nc; ++k) maxcol = std::max(maxcol, c->cstart[k + 1] - c->cstart[k]);
        int dev = 0, nsm = 0, occ = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_imp_macro<D, A, NTM>, NTM, 0);
        if (e != cudaSuccess) return e;
        const int nblk = std::max(1, std::min(nsm * std::max(occ, 1), (maxcol + NTM - 1) / NTM));
        e = cudaMemsetAsync(c->imp_bar, 0, sizeof(unsigned), c->stream);
        if (e != cudaSuccess) return e;
        int km = k_macro, ncol = nc;
        const int* cs = c->cstart_d;
        unsigned* bar = c->imp_bar;
        void* args[] = {&I, &km, &ncol, &cs, &bar};
        e = cudaLaunchCooperativeKernel((const void*)k_imp_macro<D, A, NTM>, dim3(nblk), dim3(NTM), args, 0,
                                        c->stream);
        if (e != cudaSuccess) return e;
        c->launches += 1;
    }
    // microscopic system
    const T* xi = f32 ? (const T*)c->xi_f : (const T*)c->xi_d;
    const T* w = f32 ? (const T*)c->w_f : (const T*)c->w_d;
    CellP<D, T> Q;
    Q.Nc = c->Nc;
    Q.Nv = c->Nv;
    Q.Nvp = c->Nvp;
    Q.cstride = (size_t)NA * c->Nvp;
    Q.dt = dt;
    Q.R = c->cfg.R;
    Q.Pr = c->cfg.Pr;
    Q.omega = c->cfg.omega;
    Q.mu_ref = c->mu_ref;
    Q.T_ref = c->cfg.T_ref;
    Q.fin = (const T*)fin;
    Q.fout = (T*)fout;
    Q.F = (const T*)c->flux;
    Q.AF = c->AFf;
    Q.Win = Win;
    Q.Wout = Wout;
    Q.mom = c->cmom;
    Q.par = (CellPar<T>*)c->cpar;
    Q.xi = xi;
    Q.w = w;
    Q.xp = c->xi_p;
    Q.slot = c->slot;
    Q.nslot = c->nslot;
    Q.vol = c->vol;
    Q.err = c->dev_err;
    constexpr int NT = 128;
    if (!c->mom_valid) {
        k_raw_moments<D, T, NT, VW<T>::v><<<c->Nc, NT, 0, c->stream>>>(Q);
        c->launches += 1;
    }
    k_imp_state<D, T><<<cb, 128, 0, c->stream>>>(Q, Wout);
    k_imp_res<D, T, NT, VW<T>::v><<<c->Nc, NT, 0, c->stream>>>(Q);
    c->launches += 2;
    T* dphi = (T*)c->flux;                    // the face flux has been used: its buffer holds dphi
    e = cudaMemsetAsync(dphi, 0, (size_t)c->Nc * NA * c->Nvp * sizeof(T), c->stream);
    if (e != cudaSuccess) return e;
    constexpr int VM = VW<T>::v;
    const int nyb = (c->Nv + NT * VM - 1) / (NT * VM);
    const T* Anv = f32 ? (const T*)c->An_f : (const T*)c->An_d;
    int prev = -1;
    for (int it = 0; it < k_micro; ++it)
        for (int dir = 0; dir < 2; ++dir)
            for (int q = 0; q < nc; ++q) {
                const int col = dir == 0 ? q : nc - 1 - q;
                if (col == prev) continue;      // the turn of a symmetric sweep: same inputs, same values
                prev = col;
                const int c0 = c->cstart[col], c1 = c->cstart[col + 1];
                if (c1 > c0) {
                    dim3 g(c1 - c0, nyb);
                    k_imp_micro<D, T, NT, VM><<<g, NT, 0, c->stream>>>(Q, (const T*)fout, dphi, Anv, c->faceL,
                                                                        c->faceR, c->clist, c0);
                    c->launches += 1;
                }
            }
    dim3 gf(c->Nc * NA, (c->Nvp + 255) / 256 < 8 ? (c->Nvp + 255) / 256 : 8);
    k_imp_finish<T><<<gf, 256, 0, c->stream>>>(c->Nc * NA, c->Nv, c->Nvp, (const T*)fin, dphi, (T*)fout);
    c->launches += 1;
    c->mom_valid = 0;          // the carried moments are of f^n
    (void)NW;
    return cudaGetLastError();
}

cudaError_t launch_step_implicit(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt,
                                 int k_macro, int k_micro)
{
    if (c->D == 2)
        return c->mixed ? launch_step_implicit_t<2, float>(c, fin, fout, Win, Wout, dt, k_macro, k_micro)
                        : launch_step_implicit_t<2, double>(c, fin, fout, Win, Wout, dt, k_macro, k_micro);
    return c->mixed ? launch_step_implicit_t<3, float>(c, fin, fout, Win, Wout, dt, k_macro, k_micro)
                    : launch_step_implicit_t<3, double>(c, fin, fout, Win, Wout, dt, k_macro, k_micro);
}

void launch_grad_rykov(avs_ctx* c, const void* fin)
{
    if (c->D == 2) {
        if (c->mixed) grad_t<2, float, 3>(c, fin);
        else grad_t<2, double, 3>(c, fin);
    } else {
        if (c->mixed) grad_t<3, float, 2>(c, fin);
        else grad_t<3, double, 2>(c, fin);
    }
}

cudaError_t launch_face_stage(avs_ctx* c, const void* fin, const double* Win, double dt)
{
    if (c->D == 2)
        return c->mixed ? face_stage_t<2, float>(c, fin, Win, dt) : face_stage_t<2, double>(c, fin, Win, dt);
    return c->mixed ? face_stage_t<3, float>(c, fin, Win, dt) : face_stage_t<3, double>(c, fin, Win, dt);
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
