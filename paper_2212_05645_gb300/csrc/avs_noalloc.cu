// avs_criterion_noalloc: the adaptive criterion M_k for caller-owned device
// arrays, with its scratch in fixed file-scope device arrays instead of
// memory from cudaMalloc.
//
// Why it exists: some callers cannot allocate device memory on demand.
// Examples are embedders whose device memory is owned by another allocator
// (a framework's caching pool, a fixed memory budget) and latency-sensitive
// loops that cannot pay for the device-wide synchronisation that cudaMalloc
// and cudaFree imply.  This entry point allocates nothing: the caller passes
// inputs and outputs, and the scratch lives in the arrays below, which every
// GPU that loads the library holds until the process exits.
//
// Limits: at most AVS_NOALLOC_MAX_CELLS cells (per-cell inputs, 5 doubles
// each: 10 MiB) and AVS_NOALLOC_MAX_NODES velocity nodes (ordered 64-bit keys
// for the max reduction: 1 MiB).  Larger problems get AVS_ECAPACITY.
//
// Sharing: all calls on a device share these arrays and the arrays keep the
// last call's contents; each call re-initialises what must start fresh (the
// keys are reset to the key of -infinity before the reduction).  Calls whose
// kernels overlap on the GPU (for example on two streams without ordering)
// race on the scratch and give wrong results.
//
// Set-up: the first call on each device looks up the device address of the
// scratch with cudaGetSymbolAddress (that device current) and caches it with
// the identity of the device's current context.  Make that first call before
// any stream capture begins.  A device reset (cudaDeviceReset) destroys the
// context and the module with it; the next call sees a new context identity
// and looks the address up again, so no kernel is ever given the old one.
//
// Errors: the call reports the launch status of its own kernels only; an
// error left pending by earlier code on this thread is cleared first, not
// reported as this call's failure.
#include <cuda.h>
#include <stdio.h>

#include <mutex>

#include "avs_dev.cuh"
#include "avs_internal.h"

#define AVS_NOALLOC_MAX_CELLS (1 << 18)
#define AVS_NOALLOC_MAX_NODES (1 << 17)
#define AVS_NOALLOC_MAX_DEVICES 64

namespace {

static __device__ __align__(256) double g_cell_inputs[AVS_NOALLOC_MAX_CELLS * 5];
static __device__ __align__(256) unsigned long long g_node_keys[AVS_NOALLOC_MAX_NODES];

struct ScratchAddr {
    double* cells = nullptr;
    unsigned long long* keys = nullptr;
    unsigned long long ctx_id = 0;     // context the addresses belong to (0: unknown)
};
ScratchAddr g_addr[AVS_NOALLOC_MAX_DEVICES];
std::mutex g_addr_mu;

// Unique identity of the calling thread's current context, 0 when none is
// current or the driver does not report one.  The two driver functions are
// taken through the runtime's entry-point query, so the library needs no
// link to the driver library.
unsigned long long current_context_id()
{
    typedef CUresult (*get_current_t)(CUcontext*);
    typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (get_current_t)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (get_id_t)p;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Per-cell inputs of the criterion in the fixed order of its definition:
// rho, U_d = m_d / rho, e_int = rho E - 0.5 (sum m_d m_d) / rho.
__global__ void k_na_cells(int D, int Nc, const double* __restrict__ Wc, double* cp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    const double* W = Wc + (size_t)i * (D + 2);
    const double rho = W[0];
    double mm = 0.0;
    for (int d = 0; d < D; ++d) {
        cp[(size_t)i * 5 + 1 + d] = __ddiv_rn(W[1 + d], rho);
        mm = __dadd_rn(mm, __dmul_rn(W[1 + d], W[1 + d]));
    }
    cp[(size_t)i * 5 + 0] = rho;
    cp[(size_t)i * 5 + 4] = __dsub_rn(W[D + 1], __ddiv_rn(__dmul_rn(0.5, mm), rho));
}

__global__ void k_na_fill(unsigned long long* keys, int n, unsigned long long v)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) keys[k] = v;
}

// M_k = max over cells of max((w G)/rho, ((0.5 (w G)) c^2)/e_int)
__global__ void k_na_max(int D, int NA, int Nv, int Nc, int cells_per_block, const double* __restrict__ f,
                         const double* __restrict__ xi, const double* __restrict__ w,
                         const double* __restrict__ cp, unsigned long long* keys)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Nv) return;
    const int j0 = blockIdx.y * cells_per_block;
    const int j1 = min(Nc, j0 + cells_per_block);
    double x[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) x[d] = xi[(size_t)k * D + d];
    const double wk = w[k];
    double best = -INFINITY;
    for (int i = j0; i < j1; ++i) {
        const double* p = cp + (size_t)i * 5;
        const double wg = __dmul_rn(wk, f[(size_t)i * NA * Nv + k]);
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
    if (best > -INFINITY) atomicMax(keys + k, avs::dkey(best));
}

__global__ void k_na_decode(const unsigned long long* __restrict__ keys, double* M, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) M[k] = avs::dkey_inv(keys[k]);
}

}  // namespace

extern "C" avs_status avs_criterion_noalloc(int dim, int Nc, int Nv, const double* f, const double* xi,
                                            const double* w, const double* Wc, double* M_out, void* cuda_stream)
{
    if ((dim != 2 && dim != 3) || Nc <= 0 || Nv <= 0 || !f || !xi || !w || !Wc || !M_out) {
        fprintf(stderr, "avs_criterion_noalloc: invalid argument\n");
        return AVS_EINVAL;
    }
    if (Nc > AVS_NOALLOC_MAX_CELLS || Nv > AVS_NOALLOC_MAX_NODES) {
        fprintf(stderr,
                "avs_criterion_noalloc: %d cells x %d nodes exceeds the fixed scratch (at most %d cells and %d "
                "nodes)\n",
                Nc, Nv, AVS_NOALLOC_MAX_CELLS, AVS_NOALLOC_MAX_NODES);
        return AVS_ECAPACITY;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= AVS_NOALLOC_MAX_DEVICES) return AVS_ECUDA;
    ScratchAddr a;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        const unsigned long long id = current_context_id();
        if (!g_addr[dev].cells || id == 0 || id != g_addr[dev].ctx_id) {
            void* pc = nullptr;
            void* pk = nullptr;
            if (cudaGetSymbolAddress(&pc, g_cell_inputs) != cudaSuccess ||
                cudaGetSymbolAddress(&pk, g_node_keys) != cudaSuccess) {
                fprintf(stderr, "avs_criterion_noalloc: cudaGetSymbolAddress failed\n");
                g_addr[dev] = ScratchAddr();
                return AVS_ECUDA;
            }
            g_addr[dev].cells = (double*)pc;
            g_addr[dev].keys = (unsigned long long*)pk;
            g_addr[dev].ctx_id = current_context_id();   // the lookup made the context current
        }
        a = g_addr[dev];
    }
    (void)cudaGetLastError();          // report this call's launches only
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int NA = dim == 2 ? 2 : 1;
    const int cpb = 64;
    k_na_cells<<<(Nc + 255) / 256, 256, 0, s>>>(dim, Nc, Wc, a.cells);
    k_na_fill<<<(Nv + 255) / 256, 256, 0, s>>>(a.keys, Nv, avs::dkey(-INFINITY));
    dim3 g((Nv + 255) / 256, (Nc + cpb - 1) / cpb);
    k_na_max<<<g, 256, 0, s>>>(dim, NA, Nv, Nc, cpb, f, xi, w, a.cells, a.keys);
    k_na_decode<<<(Nv + 255) / 256, 256, 0, s>>>(a.keys, M_out, Nv);
    return cudaGetLastError() == cudaSuccess ? AVS_OK : AVS_ECUDA;
}
