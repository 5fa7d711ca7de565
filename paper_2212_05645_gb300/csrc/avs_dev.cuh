// Device-side building blocks of the UGKS/AVS kernels (sm_103a).
//
// Element type T is double (FP64 form) or float (mixed form: f, reconstruction,
// flux and collision in FP32; every velocity-space sum is carried into FP64
// through short FP32 partials flushed into double accumulators).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#define AVS_MAXS 6            // face slots per cell (hexahedra)
#define AVS_PI 3.14159265358979323846

namespace avs {

template <int D> struct NArr { static constexpr int v = (D == 2) ? 2 : 1; };
// raw velocity moments of one distribution pair about a reference velocity V:
// 2D: G{1, x, y, xx, xy, yy, x s, y s} + H{1, x, y}       (s = |xi - V|^2)
// 3D: G{1, x, y, z, xx, xy, xz, yy, yz, zz, x s, y s, z s}
template <int D> struct NMom { static constexpr int v = (D == 2) ? 11 : 13; };

// ---------------------------------------------------------------- numerics
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float dmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float dadd(float a, float b) { return __fadd_rn(a, b); }

// xi . An summed left to right without fused multiply-add, so that the upwind
// choice (sign test) is made on the same value as in a plain sequential code.
template <int D, typename T>
__device__ __forceinline__ T dot_rn(const T* x, const T* a)
{
    T s = dmul(x[0], a[0]);
    s = dadd(s, dmul(x[1], a[1]));
    if (D == 3) s = dadd(s, dmul(x[2], a[2]));
    return s;
}

// exp: correctly rounded library exp in FP64; the hardware ex2 path in the
// FP32 form (relative error a few ulp, far below the FP32 storage of f).
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex(float x) { return __expf(x); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }

// ---------------------------------------------------------------- geometry
template <typename T>
struct CellGeo {
    const int* __restrict__ nbr;            // [Nc][MAXS] neighbour cell, -1 none/boundary
    const T* __restrict__ cg;               // [Nc][MAXS][D] least-squares weights
    const T* __restrict__ r;                // [Nc][MAXS][D] face centre - cell centre
    const T* __restrict__ eps2;             // [Nc] Venkatakrishnan eps^2
    const unsigned char* __restrict__ ns;   // [Nc] number of face slots
};

// ---------------------------------------------------------------- bulk copies
// Asynchronous 1D bulk copies global -> shared memory that complete on an
// mbarrier (transaction count in bytes).  Addresses and sizes must be
// multiples of 16 bytes; callers guarantee it by construction.
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the asynchronous (copy) proxy
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// orders this thread's earlier generic-proxy accesses of shared memory before
// later asynchronous-proxy writes (a buffer refilled after it was read)
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Waits for the barrier's phase of the given parity, for at most about
// `cycles` SM clock cycles; false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long cycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}

// Largest / smallest of three values (PTX three-input max / min on FP32;
// exact, like the two-input forms).
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Venkatakrishnan limiter function, capped at 1.
template <typename T>
__device__ __forceinline__ T venkat(T d1, T d2, T eps2)
{
    T num = d1 * d1 + eps2 + T(2) * d1 * d2;
    T den = d1 * d1 + T(2) * d2 * d2 + d1 * d2 + eps2;
    T v = fdiv(num, den);
    return v < T(1) ? v : T(1);
}

// log2(e), and log2 in the argument's type
constexpr double kLog2e = 1.4426950408889634;
__device__ __forceinline__ double log2a(double x) { return log2(x); }
__device__ __forceinline__ float log2a(float x) { return log2f(x); }
// 2^x by the PTX ex2 instruction (approximate, subnormal results flushed to zero)
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------- equilibria
// Parameters of one equilibrium evaluated on the nodes:
//   G = pref exp(-|c|^2 inv2RT) (1 + (c . alpha)(|c|^2 invRT - D - 2)),
//   H = RTH exp(..)pref (1 + (c . alpha)(|c|^2 invRT - D)),   c = xi - U
// which is the Shakhov form of Eqs. 14-17 (K = 0) with
// alpha = (1 - Pr) q / (5 p R T), and the plain Maxwellian when alpha = 0.
template <typename T>
struct EqPar {
    T pref, U[3], inv2RT, invRT, RTH, alpha[3];
    T l2pref, k2;            // log2(pref) and -log2(e) / (2 R T): the FP32 pair form's base-2 exponent
};

template <int D, typename T>
__device__ __forceinline__ void eq_eval(const EqPar<T>& p, const T* x, T& gG, T& gH)
{
    T c[D];
    T c2 = T(0), cq = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        c[d] = x[d] - p.U[d];
        c2 += c[d] * c[d];
        cq += c[d] * p.alpha[d];
    }
    const T e = p.pref * ex(-c2 * p.inv2RT);
    const T s = c2 * p.invRT;
    gG = e * (T(1) + cq * (s - T(D + 2)));
    gH = (D == 2) ? p.RTH * e * (T(1) + cq * (s - T(D))) : T(0);
}

// Host/device: equilibrium parameters from rho, U, RT, q (double inputs).
template <int D, typename T>
__device__ __forceinline__ EqPar<T> make_eq(double rho, const double* U, double RT, const double* q,
                                            double Pr)
{
    EqPar<T> p;
    const double t = 2.0 * AVS_PI * RT;
    const double pref = rho / (D == 2 ? t : t * sqrt(t));
    p.pref = (T)pref;
    const double a = (1.0 - Pr) / (5.0 * rho * RT * RT);
    for (int d = 0; d < 3; ++d) {
        p.U[d] = d < D ? (T)U[d] : T(0);
        p.alpha[d] = (d < D && q) ? (T)(a * q[d]) : T(0);
    }
    p.inv2RT = (T)(1.0 / (2.0 * RT));
    p.invRT = (T)(1.0 / RT);
    p.RTH = (T)((3.0 - D) * RT);
    p.l2pref = (T)log2(pref);
    p.k2 = (T)(-kLog2e / (2.0 * RT));
    return p;
}

// conserved (rho, m, E) -> rho, U, RT (monatomic: E = m^2/2rho + 3/2 rho R T)
template <int D>
__device__ __forceinline__ void prim(const double* Wc, double& rho, double* U, double& RT)
{
    rho = Wc[0];
    double m2 = 0.0;
    for (int d = 0; d < D; ++d) {
        U[d] = Wc[1 + d] / rho;
        m2 += Wc[1 + d] * Wc[1 + d];
    }
    RT = (Wc[D + 1] - 0.5 * m2 / rho) / (1.5 * rho);
}

// ---------------------------------------------------------------- moments
// Accumulate the raw-moment contributions of one node (weight already folded
// into wg, wh) about reference velocity; xs = xi - V.
template <int D, typename T>
__device__ __forceinline__ void raw_acc(T* m, const T* xs, T wg, T wh)
{
    if (D == 2) {
        const T s = xs[0] * xs[0] + xs[1] * xs[1];
        m[0] += wg;
        m[1] += wg * xs[0];
        m[2] += wg * xs[1];
        m[3] += wg * xs[0] * xs[0];
        m[4] += wg * xs[0] * xs[1];
        m[5] += wg * xs[1] * xs[1];
        m[6] += wg * xs[0] * s;
        m[7] += wg * xs[1] * s;
        m[8] += wh;
        m[9] += wh * xs[0];
        m[10] += wh * xs[1];
    } else {
        const T s = xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2];
        m[0] += wg;
        m[1] += wg * xs[0];
        m[2] += wg * xs[1];
        m[3] += wg * xs[2];
        m[4] += wg * xs[0] * xs[0];
        m[5] += wg * xs[0] * xs[1];
        m[6] += wg * xs[0] * xs[2];
        m[7] += wg * xs[1] * xs[1];
        m[8] += wg * xs[1] * xs[2];
        m[9] += wg * xs[2] * xs[2];
        m[10] += wg * xs[0] * s;
        m[11] += wg * xs[1] * s;
        m[12] += wg * xs[2] * s;
    }
}

// Raw moments about V (m) -> conserved W, heat flux q about the own mean
// velocity (Eq. 8), and optionally the area-weighted flux of W through An:
// A F = sum_k w (xi . An) (G, xi G, (|xi|^2 G + H)/2).
template <int D>
__device__ void moments_from_raw(const double* m, const double* V, double* W, double* q,
                                 const double* An, double* AF)
{
    // shifted moments S0, S1[a], S2[a][b], S3[a] (S3 = sum w x_a |x|^2 G), H0, H1[a]
    double S0 = m[0], S1[3], S2[3][3], S3[3], H0 = 0, H1[3] = {0, 0, 0};
    if (D == 2) {
        S1[0] = m[1]; S1[1] = m[2];
        S2[0][0] = m[3]; S2[0][1] = S2[1][0] = m[4]; S2[1][1] = m[5];
        S3[0] = m[6]; S3[1] = m[7];
        H0 = m[8]; H1[0] = m[9]; H1[1] = m[10];
    } else {
        S1[0] = m[1]; S1[1] = m[2]; S1[2] = m[3];
        S2[0][0] = m[4]; S2[0][1] = S2[1][0] = m[5]; S2[0][2] = S2[2][0] = m[6];
        S2[1][1] = m[7]; S2[1][2] = S2[2][1] = m[8]; S2[2][2] = m[9];
        S3[0] = m[10]; S3[1] = m[11]; S3[2] = m[12];
    }
    double trS2 = 0.0;
    for (int a = 0; a < D; ++a) trS2 += S2[a][a];
    // conserved variables
    double rho = S0;
    double d[3];                   // mean velocity relative to V
    for (int a = 0; a < D; ++a) d[a] = S1[a] / rho;
    W[0] = rho;
    double V2 = 0.0, VS1 = 0.0;
    for (int a = 0; a < D; ++a) { V2 += V[a] * V[a]; VS1 += V[a] * S1[a]; }
    for (int a = 0; a < D; ++a) W[1 + a] = S1[a] + rho * V[a];
    W[D + 1] = 0.5 * (trS2 + 2.0 * VS1 + rho * V2 + H0);
    // heat flux about U = V + d:  1/2 sum w c_a (|c|^2 G + H), c = x' - d
    if (q) {
        double dd = 0.0;
        for (int a = 0; a < D; ++a) dd += d[a] * d[a];
        for (int a = 0; a < D; ++a) {
            double S2d = 0.0;
            for (int b = 0; b < D; ++b) S2d += S2[a][b] * d[b];
            double dS1 = 0.0;
            for (int b = 0; b < D; ++b) dS1 += d[b] * S1[b];
            double g3 = S3[a] - 2.0 * S2d + dd * S1[a] - d[a] * trS2 + 2.0 * d[a] * dS1 - d[a] * dd * S0;
            double h1 = H1[a] - d[a] * H0;
            q[a] = 0.5 * (g3 + h1);
        }
    }
    if (AF) {
        // flux moments of the raw (unshifted) distribution through An
        double Fm = 0.0;
        for (int a = 0; a < D; ++a) Fm += An[a] * (S1[a] + rho * V[a]);
        AF[0] = Fm;
        for (int b = 0; b < D; ++b) {
            double s = 0.0;
            for (int a = 0; a < D; ++a)
                s += An[a] * (S2[a][b] + V[a] * S1[b] + S1[a] * V[b] + rho * V[a] * V[b]);
            AF[1 + b] = s;
        }
        double E = 0.0;
        for (int a = 0; a < D; ++a) {
            double S2V = 0.0;
            for (int b = 0; b < D; ++b) S2V += S2[a][b] * V[b];
            double g = S3[a] + 2.0 * S2V + V2 * S1[a] + V[a] * trS2 + 2.0 * V[a] * VS1 + V[a] * V2 * S0;
            double h = H1[a] + V[a] * H0;
            E += An[a] * (g + h);
        }
        AF[D + 1] = 0.5 * E;
    }
}

// Raw moments about V (m, FP64 sums) -> rho, U, RT and heat flux q about the
// own mean velocity, evaluated in type A.  With V close to the mean velocity
// the shifted moments are nearly central, so no large terms cancel:
// e_int = (tr S2 + H0)/2 - rho |d|^2 / 2, d = S1 / rho (3/2 rho R T, monatomic).
template <int D, typename A>
__device__ __forceinline__ void state_from_raw(const double* m, const double* V, A& rho, A* U, A& RT, A* q)
{
    A S1[3], S2[3][3], S3[3], H0 = A(0), H1[3] = {A(0), A(0), A(0)};
    const A S0 = (A)m[0];
    if (D == 2) {
        S1[0] = (A)m[1]; S1[1] = (A)m[2];
        S2[0][0] = (A)m[3]; S2[0][1] = S2[1][0] = (A)m[4]; S2[1][1] = (A)m[5];
        S3[0] = (A)m[6]; S3[1] = (A)m[7];
        H0 = (A)m[8]; H1[0] = (A)m[9]; H1[1] = (A)m[10];
    } else {
        S1[0] = (A)m[1]; S1[1] = (A)m[2]; S1[2] = (A)m[3];
        S2[0][0] = (A)m[4]; S2[0][1] = S2[1][0] = (A)m[5]; S2[0][2] = S2[2][0] = (A)m[6];
        S2[1][1] = (A)m[7]; S2[1][2] = S2[2][1] = (A)m[8]; S2[2][2] = (A)m[9];
        S3[0] = (A)m[10]; S3[1] = (A)m[11]; S3[2] = (A)m[12];
    }
    rho = S0;
    const A ir = fdiv(A(1), S0);
    A d[3], dd = A(0), trS2 = A(0), dS1 = A(0);
    for (int a = 0; a < D; ++a) {
        d[a] = S1[a] * ir;
        U[a] = (A)V[a] + d[a];
        dd += d[a] * d[a];
        trS2 += S2[a][a];
        dS1 += d[a] * S1[a];
    }
    RT = fdiv(A(0.5) * (trS2 + H0) - A(0.5) * S0 * dd, A(1.5) * S0);
    if (q) {
        for (int a = 0; a < D; ++a) {
            A S2d = A(0);
            for (int b = 0; b < D; ++b) S2d += S2[a][b] * d[b];
            const A g3 = S3[a] - A(2) * S2d + dd * S1[a] - d[a] * trS2 + A(2) * d[a] * dS1 - d[a] * dd * S0;
            q[a] = A(0.5) * (g3 + H1[a] - d[a] * H0);
        }
    }
}

// Equilibrium parameters from rho, U, RT, q given in type A.
template <int D, typename T, typename A>
__device__ __forceinline__ EqPar<T> make_eq_a(A rho, const A* U, A RT, const A* q, A Pr)
{
    EqPar<T> p;
    const A t = A(2.0 * AVS_PI) * RT;
    p.pref = (T)fdiv(rho, D == 2 ? t : t * sqrt(t));
    const A a = fdiv(A(1) - Pr, A(5) * rho * RT * RT);
    for (int d = 0; d < 3; ++d) {
        p.U[d] = d < D ? (T)U[d] : T(0);
        p.alpha[d] = (d < D && q) ? (T)(a * q[d]) : T(0);
    }
    p.inv2RT = (T)fdiv(A(1), A(2) * RT);
    p.invRT = (T)fdiv(A(1), RT);
    p.RTH = (T)(A(3 - D) * RT);
    p.l2pref = (T)log2a(fdiv(rho, D == 2 ? t : t * sqrt(t)));
    p.k2 = (T)(-A(kLog2e) * fdiv(A(1), A(2) * RT));
    return p;
}

__device__ __forceinline__ double powa(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float powa(float x, float y) { return exp2f(y * __log2f(x)); }

// ---------------------------------------------------------------- vector access
// N consecutive elements starting at a 16-byte aligned address, moved as
// 16-byte vectors (N * sizeof(T) a multiple of 16).
template <typename T, int N>
__device__ __forceinline__ void vload(const T* __restrict__ p, T* o)
{
    static_assert((N * sizeof(T)) % 16 == 0, "whole 16-byte vectors");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int j = 0; j < N / 4; ++j) {
            const float4 q = reinterpret_cast<const float4*>(p)[j];
            o[4 * j] = q.x; o[4 * j + 1] = q.y; o[4 * j + 2] = q.z; o[4 * j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            const double2 q = reinterpret_cast<const double2*>(p)[j];
            o[2 * j] = q.x; o[2 * j + 1] = q.y;
        }
    }
}

template <typename T, int N>
__device__ __forceinline__ void vstore(T* p, const T* o)
{
    static_assert((N * sizeof(T)) % 16 == 0, "whole 16-byte vectors");
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int j = 0; j < N / 4; ++j)
            reinterpret_cast<float4*>(p)[j] = make_float4(o[4 * j], o[4 * j + 1], o[4 * j + 2], o[4 * j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < N / 2; ++j) reinterpret_cast<double2*>(p)[j] = make_double2(o[2 * j], o[2 * j + 1]);
    }
}

// ---------------------------------------------------------------- criterion screening
// FP32 screening value of the criterion at one (cell, node), scaled by 2^64,
// and a bound on its distance from the exact value times 2^64.  The scaling
// (exact, a power of two applied to G) keeps the FP32 values of the small f of
// the distribution tails in the normal range.  With xi, U, w, G, 1/rho,
// 0.5/e_int and every operation rounded to FP32 (u = 2^-24) and normal results:
//   |M1_32 - M1| <= 6 u |M1|;
//   |c_d,32 - c_d| <= delta_d = u a_d + 1.01 u |c_d|,  a_d = |xi_d| + |U_d|,
//   |c^2_32 - c^2| <= sum_d delta_d (2 |c_d| + delta_d) + 4 u c^2,
//   |M2_32 - M2| <= |wG 0.5/e| (16 u sum_d a_d |c_d| + 16 u^2 sum_d a_d^2 + 44 u c^2).
// The bound takes 128 u for the first-order terms and 2^-40 for the
// second-order one, and adds 2^-126, the smallest normal FP32 number, which
// covers the absolute error of the roundings that can still fall in the
// subnormal range (2^-150 each).
constexpr float kCritScale = 0x1p64f;

// G * 2^64 in FP32 (the scaling done in the type of G, so no extra underflow)
__device__ __forceinline__ float crit_scaled(float G) { return G * kCritScale; }
__device__ __forceinline__ float crit_scaled(double G) { return (float)(G * 0x1p64); }

__device__ __forceinline__ void crit32(int D, float Gs, float wk, const float* x, const float* c32, float& m, float& B)
{
    const float wg = wk * Gs;
    const float m1 = wg * c32[0];
    float c2 = 0.0f, ac = 0.0f, a2 = 0.0f;
    for (int d = 0; d < D; ++d) {
        const float cc = x[d] - c32[1 + d];
        const float aa = fabsf(x[d]) + fabsf(c32[1 + d]);
        c2 += cc * cc;
        ac += aa * fabsf(cc);
        a2 += aa * aa;
    }
    const float wh = wg * c32[4];
    const float m2 = wh * c2;
    m = m1 > m2 ? m1 : m2;
    const float awh = fabsf(wh);
    B = 0x1p-17f * (fabsf(m1) + awh * (ac + c2)) + 0x1p-40f * awh * a2 + 0x1p-126f;
}

// ---------------------------------------------------------------- FP32 pairs
// Two nodes per instruction with the packed two-lane FP32 operations of
// sm_100+ (each lane rounds as the scalar operation does; no contraction
// beyond the explicit fma2).
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Compensated FP32 accumulation: s + c carries the running sum, c the exact
// rounding errors of the additions (TwoSum, no multiply so no contraction), so
// a per-thread sum of FP32 terms keeps about twice the FP32 precision.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float y)
{
    const float t = s + y;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (y - bp);
    s = t;
    c += e;
}

// raw_acc with compensated per-thread sums (s, c) of the same terms.
template <int D>
__device__ __forceinline__ void raw_acc_c(float* s, float* c, const float* xs, float wg, float wh)
{
    if (D == 2) {
        const float q = xs[0] * xs[0] + xs[1] * xs[1];
        const float t0 = wg * xs[0], t1 = wg * xs[1];
        two_sum_acc(s[0], c[0], wg);
        two_sum_acc(s[1], c[1], t0);
        two_sum_acc(s[2], c[2], t1);
        two_sum_acc(s[3], c[3], t0 * xs[0]);
        two_sum_acc(s[4], c[4], t0 * xs[1]);
        two_sum_acc(s[5], c[5], t1 * xs[1]);
        two_sum_acc(s[6], c[6], t0 * q);
        two_sum_acc(s[7], c[7], t1 * q);
        two_sum_acc(s[8], c[8], wh);
        two_sum_acc(s[9], c[9], wh * xs[0]);
        two_sum_acc(s[10], c[10], wh * xs[1]);
    } else {
        const float q = xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2];
        const float t0 = wg * xs[0], t1 = wg * xs[1], t2 = wg * xs[2];
        two_sum_acc(s[0], c[0], wg);
        two_sum_acc(s[1], c[1], t0);
        two_sum_acc(s[2], c[2], t1);
        two_sum_acc(s[3], c[3], t2);
        two_sum_acc(s[4], c[4], t0 * xs[0]);
        two_sum_acc(s[5], c[5], t0 * xs[1]);
        two_sum_acc(s[6], c[6], t0 * xs[2]);
        two_sum_acc(s[7], c[7], t1 * xs[1]);
        two_sum_acc(s[8], c[8], t1 * xs[2]);
        two_sum_acc(s[9], c[9], t2 * xs[2]);
        two_sum_acc(s[10], c[10], t0 * q);
        two_sum_acc(s[11], c[11], t1 * q);
        two_sum_acc(s[12], c[12], t2 * q);
    }
}

// raw_acc for a pair of nodes (per-lane partial sums), D = 2 or 3
template <int D>
__device__ __forceinline__ void raw_acc2(float2* m, const float2* xs, float2 wg, float2 wh)
{
    if (D == 2) {
        const float2 s = fma2(xs[1], xs[1], mul2(xs[0], xs[0]));
        const float2 t0 = mul2(wg, xs[0]), t1 = mul2(wg, xs[1]);
        m[0] = add2(m[0], wg);
        m[1] = add2(m[1], t0);
        m[2] = add2(m[2], t1);
        m[3] = fma2(t0, xs[0], m[3]);
        m[4] = fma2(t0, xs[1], m[4]);
        m[5] = fma2(t1, xs[1], m[5]);
        m[6] = fma2(t0, s, m[6]);
        m[7] = fma2(t1, s, m[7]);
        m[8] = add2(m[8], wh);
        m[9] = fma2(wh, xs[0], m[9]);
        m[10] = fma2(wh, xs[1], m[10]);
    } else {
        const float2 s = fma2(xs[2], xs[2], fma2(xs[1], xs[1], mul2(xs[0], xs[0])));
        const float2 t0 = mul2(wg, xs[0]), t1 = mul2(wg, xs[1]), t2 = mul2(wg, xs[2]);
        m[0] = add2(m[0], wg);
        m[1] = add2(m[1], t0);
        m[2] = add2(m[2], t1);
        m[3] = add2(m[3], t2);
        m[4] = fma2(t0, xs[0], m[4]);
        m[5] = fma2(t0, xs[1], m[5]);
        m[6] = fma2(t0, xs[2], m[6]);
        m[7] = fma2(t1, xs[1], m[7]);
        m[8] = fma2(t1, xs[2], m[8]);
        m[9] = fma2(t2, xs[2], m[9]);
        m[10] = fma2(t0, s, m[10]);
        m[11] = fma2(t1, s, m[11]);
        m[12] = fma2(t2, s, m[12]);
    }
}

// eq_eval for a pair of nodes (X[d] = the pair's d-th velocity components)
template <int D>
__device__ __forceinline__ void eq_eval2(const EqPar<float>& p, const float2* X, float2& gG, float2& gH)
{
    float2 c[D];
#pragma unroll
    for (int d = 0; d < D; ++d) c[d] = add2(X[d], bc2(-p.U[d]));
    float2 c2 = mul2(c[0], c[0]), cq = mul2(c[0], bc2(p.alpha[0]));
#pragma unroll
    for (int d = 1; d < D; ++d) {
        c2 = fma2(c[d], c[d], c2);
        cq = fma2(c[d], bc2(p.alpha[d]), cq);
    }
    // pref exp(-c^2 / 2RT) as 2^(log2 pref - c^2 log2(e) / 2RT): one fused
    // multiply-add for the exponent of both lanes
    const float2 a = fma2(c2, bc2(p.k2), bc2(p.l2pref));
    const float2 e = make_float2(ex2_approx(a.x), ex2_approx(a.y));
    const float2 s = mul2(c2, bc2(p.invRT));
    gG = mul2(e, fma2(cq, add2(s, bc2(-(float)(D + 2))), bc2(1.0f)));
    gH = (D == 2) ? mul2(mul2(bc2(p.RTH), e), fma2(cq, add2(s, bc2(-(float)D)), bc2(1.0f))) : bc2(0.0f);
}

// ---------------------------------------------------------------- reductions
// Deterministic block reduction of N doubles per thread: warp tree with
// shuffles, then a fixed-order sum over warps.  Result in out[0..N-1] (smem),
// visible to all threads after return.
template <int N, int NT>
__device__ __forceinline__ void block_sum(double* v, double* sred, double* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < N; ++m) {
        double x = v[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sred[warp * N + m] = x;
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += sred[w * N + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// float -> double by bit manipulation on the integer pipe (exact for normal
// numbers; subnormals, far below any partial sum here, become signed zero).
// On GB300 the FP64 pipe, which executes the usual conversion, is scarce.
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned sgn = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    unsigned hi, lo;
    if (e == 0u) {
        hi = sgn;
        lo = 0u;
    } else if (e == 0xFFu) {
        hi = sgn | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else {
        hi = sgn | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// Block reduction of N values per thread kept in the element type: warp tree
// with shuffles in T, then a fixed-order FP64 sum of the per-warp results.
// Deterministic.  out[0..N-1] (smem, double) is visible to all threads after
// return.  sw must hold (NT/32)*N doubles.
template <int N, int NT, typename T>
__device__ __forceinline__ void block_sum_t(T* v, double* sw, double* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 0; m < N; ++m) {
        T x = v[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sw[warp * N + m] = to_double(x);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < N; m += NT) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += sw[w * N + m];
        out[m] = s;
    }
    __syncthreads();
}

// Ordered 64-bit key of a double (monotone for all finite values) for
// atomicMax/atomicMin on doubles.
__host__ __device__ __forceinline__ unsigned long long dkey(double x)
{
    unsigned long long b;
    memcpy(&b, &x, sizeof(b));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double dkey_inv(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double x;
    memcpy(&x, &b, sizeof(x));
    return x;
}

// Grid-wide barrier of a cooperative launch, bounded: the block's thread 0
// counts in and waits for the target count at most kGridSpin polls; a timeout
// (or one seen in another block) sets error bit 2 and makes the block leave.
// Monotone counter: the n-th barrier waits for n * gridDim.x arrivals.
constexpr long long kGridSpin = 1ll << 21;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar, unsigned target, int* err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int good = 1;
        for (long long it = 0; ld_acquire_u32(bar) < target; ++it) {
            if (it >= kGridSpin || ((it & 255) == 255 && (*(volatile int*)err & 2))) {
                atomicOr(err, 2);
                good = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace avs
