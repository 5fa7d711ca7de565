// C ABI of the library (include/avs.h): validation, mesh preprocessing,
// the step-0 velocity mesh, state management and every entry point.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "avs_dev.cuh"
#include "avs_internal.h"
#include "avs_mlp.h"

using namespace avs;

namespace {

avs_status fail(avs_ctx* c, avs_status s, const char* what, cudaError_t e = cudaSuccess)
{
    if (c) {
        c->err = what;
        if (e != cudaSuccess) {
            c->err += ": ";
            c->err += cudaGetErrorString(e);
        }
    }
    return s;
}

#define CK(x)                                                              \
    do {                                                                   \
        cudaError_t e_ = (x);                                              \
        if (e_ != cudaSuccess) return fail(c, AVS_ECUDA, #x, e_);          \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t n)
{
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, n * sizeof(T));
}

template <typename T>
cudaError_t up(T* dst, const std::vector<T>& v, cudaStream_t s)
{
    return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

size_t elem_size(const avs_ctx* c) { return c->mixed ? sizeof(float) : sizeof(double); }

void free_all(avs_ctx* c)
{
    void* ptrs[] = {c->faceL, c->faceR, c->An_d, c->rL_d, c->rR_d, c->An_f, c->rL_f, c->rR_f, c->vol, c->bc,
                    c->slot, c->nslot, c->nbr, c->cg_d, c->r_d, c->eps2_d, c->cg_f, c->r_f, c->eps2_f,
                    c->level, c->base, c->key, c->level2, c->base2, c->key2, c->src, c->kind, c->emit,
                    c->newidx, c->d_count, c->xi_d, c->w_d, c->xi_f, c->w_f, c->xi_p, c->M, c->Mkey, c->f[0], c->f[1],
                    c->W[0], c->W[1], c->ncap, c->Wf, c->q, c->pseudo_f, c->pseudo_W, c->crit_cp, c->crit_cp32, c->Mlo, c->Mhi, c->Mthr, c->stage, c->dev_err,
                    c->dt_key, c->gap_d, c->grad, c->flux, c->AFf, c->forder, c->cmom, c->rmom, c->cpar, c->clist, c->cstart_d, c->imp_dW, c->imp_rhs0, c->imp_diag, c->imp_Wta,
                    c->imp_co, c->imp_nint, c->imp_bar, c->mlp_P, c->mlp_Wb, c->mlp_part, c->mlp_grad,
                    c->mlp_X, c->mlp_Y, c->mlp_logits, c->mlp_list, c->mlp_count, c->M_alt};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// conserved from primitive (monatomic): rho E = rho U^2 / 2 + 3/2 rho R T
void cons_host(int D, const double* Wp, double R, double* Wc)
{
    const double rho = Wp[0];
    double u2 = 0.0;
    Wc[0] = rho;
    for (int d = 0; d < D; ++d) {
        Wc[1 + d] = rho * Wp[1 + d];
        u2 += Wp[1 + d] * Wp[1 + d];
    }
    Wc[D + 1] = 0.5 * rho * u2 + 1.5 * rho * R * Wp[D + 1];
}

// primitive (rho, U, T) from conserved W (monatomic: rho E = rho U^2 / 2 + 3/2 rho R T)
__global__ void k_cons_to_prim(int D, int Nc, const double* __restrict__ Wc, double R, double* Wp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    const double* C = Wc + (size_t)i * (D + 2);
    double* P = Wp + (size_t)i * (D + 2);
    double m2 = 0.0;
    P[0] = C[0];
    for (int d = 0; d < D; ++d) {
        P[1 + d] = C[1 + d] / C[0];
        m2 += C[1 + d] * C[1 + d];
    }
    P[D + 1] = (C[D + 1] - 0.5 * m2 / C[0]) / (1.5 * C[0] * R);
}

__global__ void k_prim_to_cons(int D, int Nc, const double* __restrict__ Wp, double R, double* Wc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nc) return;
    const double* P = Wp + (size_t)i * (D + 2);
    double* C = Wc + (size_t)i * (D + 2);
    double u2 = 0.0;
    C[0] = P[0];
    for (int d = 0; d < D; ++d) {
        C[1 + d] = P[0] * P[1 + d];
        u2 += P[1 + d] * P[1 + d];
    }
    C[D + 1] = 0.5 * P[0] * u2 + 1.5 * P[0] * R * P[D + 1];
}

avs_status read_err(avs_ctx* c)
{
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e & 4) {
        CK(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
        return fail(c, AVS_ETIMEOUT, "an asynchronous copy into the face kernel's shared memory did not complete");
    }
    if (e & 2) {
        CK(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
        return fail(c, AVS_ETIMEOUT, "a grid barrier of the implicit macroscopic sweep gave up");
    }
    if (e & 1) {
        CK(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
        return fail(c, AVS_ENUMERIC, "non-positive density or temperature in a step");
    }
    return AVS_OK;
}

avs_status refresh_dt(avs_ctx* c)
{
    CK(launch_dt_unit(c));
    unsigned long long k = 0;
    CK(cudaMemcpyAsync(&k, c->dt_key, sizeof(k), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->dt_unit = (k == ~0ull) ? INFINITY : dkey_inv(k);
    return AVS_OK;
}

// One pass of marks + compaction on criterion values already in c->M;
// swaps in the new tree.  Returns counts through out pointers.
avs_status apply_marks(avs_ctx* c, int* Nv_new, int* splits, int* merges, int uniform)
{
    CK(launch_adapt_tree(c, c->cfg.C1, c->cfg.C2, uniform));
    int cnt[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(cnt, c->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *Nv_new = cnt[0];
    *splits = cnt[1];
    *merges = cnt[2];
    if (cnt[0] > c->cap) return fail(c, AVS_ECAPACITY, "adapted velocity tree exceeds its capacity");
    return AVS_OK;
}

void swap_tree(avs_ctx* c, int Nv_new)
{
    std::swap(c->level, c->level2);
    std::swap(c->base, c->base2);
    std::swap(c->key, c->key2);
    c->Nv = Nv_new;
    c->Nvp = round_up(Nv_new, 32);
}

avs_status ensure_stage(avs_ctx* c)
{
    const size_t need = (size_t)c->Nc * c->NA * std::max(c->Nv, 1);
    if (c->stage_elems >= need) return AVS_OK;
    if (c->stage) CK(cudaFree(c->stage));
    c->stage = nullptr;
    c->stage_elems = 0;
    if (dalloc(&c->stage, need) != cudaSuccess) return fail(c, AVS_ENOMEM, "staging buffer");
    c->stage_elems = need;
    return AVS_OK;
}

avs_status alloc_f(avs_ctx* c, int nodes, void** f0, void** f1)
{
    const size_t bytes = (size_t)c->Nc * c->NA * (size_t)round_up(nodes, 32) * elem_size(c);
    if (cudaMalloc(f0, bytes) != cudaSuccess) return fail(c, AVS_ENOMEM, "f buffer");
    if (cudaMalloc(f1, bytes) != cudaSuccess) {
        cudaFree(*f0);
        return fail(c, AVS_ENOMEM, "f buffer");
    }
    CK(cudaMemsetAsync(*f0, 0, bytes, c->stream));
    CK(cudaMemsetAsync(*f1, 0, bytes, c->stream));
    return AVS_OK;
}

// He-uniform initial MLP weights from SplitMix64 (deterministic), zero biases.
void mlp_default_params(std::vector<float>& P)
{
    P.assign(AVS_MLP_NPARAM, 0.0f);
    uint64_t st = 0x5EED2212ull;
    auto uni = [&st]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1p-53;
    };
    auto fill = [&](int off, int n, int fan_in) {
        const double b = sqrt(6.0 / fan_in);
        for (int k = 0; k < n; ++k) P[off + k] = (float)((2.0 * uni() - 1.0) * b);
    };
    fill(0, 64 * 8, 8);
    fill(64 * 8 + 64, 64 * 64, 64);
    fill(64 * 8 + 64 + 64 * 64 + 64, 4 * 64, 64);
}

avs_status ensure_mlp(avs_ctx* c, int rows)
{
    if (c->mlp_P && rows <= c->mlp_rows) return AVS_OK;
    const int nrows = std::max(rows, std::max(c->Nc, 1024));
    if (!c->mlp_P) {
        if (dalloc(&c->mlp_P, AVS_MLP_NPARAM) || cudaMalloc(&c->mlp_Wb, AVS_MLP_BF16_ELEMS * 2) ||
            dalloc(&c->mlp_part, (size_t)AVS_MLP_MAXBLK * (AVS_MLP_NPARAM + 1)) ||
            dalloc(&c->mlp_grad, AVS_MLP_NPARAM + 1) || dalloc(&c->mlp_count, 2) ||
            dalloc(&c->M_alt, round_up(c->cap, 32)))
            return fail(c, AVS_ENOMEM, "MLP buffers");
        std::vector<float> P;
        mlp_default_params(P);
        CK(cudaMemcpyAsync(c->mlp_P, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(mlp_prep(c));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (c->mlp_X) { cudaFree(c->mlp_X); cudaFree(c->mlp_Y); cudaFree(c->mlp_logits); cudaFree(c->mlp_list); }
    c->mlp_X = c->mlp_Y = c->mlp_logits = nullptr;
    c->mlp_list = nullptr;
    if (dalloc(&c->mlp_X, (size_t)nrows * 8) || dalloc(&c->mlp_Y, (size_t)nrows * 4) ||
        dalloc(&c->mlp_logits, (size_t)nrows * 4) || dalloc(&c->mlp_list, nrows))
        return fail(c, AVS_ENOMEM, "MLP buffers");
    c->mlp_rows = nrows;
    return AVS_OK;
}

avs_status validate(const avs_config* cfg, const avs_mesh* m, std::string& why)
{
    if (!cfg || !m) { why = "null config or mesh"; return AVS_EINVAL; }
    const int D = cfg->dim;
    if (D != 2 && D != 3) { why = "dim must be 2 or 3"; return AVS_EINVAL; }
    if (m->dim != D) { why = "mesh dim differs from config dim"; return AVS_EINVAL; }
    if (cfg->max_refine < 0 || D * cfg->max_refine > 30) { why = "max_refine out of range"; return AVS_EINVAL; }
    long long nbase = 1;
    for (int d = 0; d < D; ++d) {
        if (cfg->base[d] < 1 || !(cfg->vhi[d] > cfg->vlo[d])) { why = "bad velocity base/bounds"; return AVS_EINVAL; }
        nbase *= cfg->base[d];
    }
    if (nbase > (1 << 24)) { why = "base forest too large"; return AVS_EINVAL; }
    if (cfg->precision != AVS_FP64 && cfg->precision != AVS_MIXED) { why = "bad precision"; return AVS_EINVAL; }
    if (!(cfg->R > 0) || !(cfg->Kn > 0) || !(cfg->T_ref > 0) || !(cfg->Pr > 0)) { why = "bad gas constants"; return AVS_EINVAL; }
    if (!(cfg->C1 > cfg->C2)) { why = "C1 must exceed C2"; return AVS_EINVAL; }
    if (cfg->limiter < 0 || cfg->limiter > 2) { why = "bad limiter"; return AVS_EINVAL; }
    if (cfg->corr_iters < 0 || cfg->corr_iters > 64) { why = "bad corr_iters"; return AVS_EINVAL; }
    if (cfg->nzones < 0 || cfg->nzones > AVS_MAX_ZONES) { why = "nzones out of range"; return AVS_EINVAL; }
    if (cfg->nzones > 0 && (cfg->zone_outside_level < 0 || cfg->zone_outside_level > cfg->max_refine)) {
        why = "zone_outside_level out of range";
        return AVS_EINVAL;
    }
    for (int z = 0; z < cfg->nzones; ++z) {
        const avs_zone& Z = cfg->zones[z];
        if (Z.level < 0 || Z.level > cfg->max_refine) { why = "zone level out of range"; return AVS_EINVAL; }
        if (!(Z.r_in >= 0) || !(Z.r_out > Z.r_in)) { why = "zone radii must satisfy 0 <= r_in < r_out"; return AVS_EINVAL; }
        for (int d = 0; d < D; ++d)
            if (!std::isfinite(Z.c[d])) { why = "zone centre not finite"; return AVS_EINVAL; }
    }
    if (cfg->init_refine < 0 || cfg->init_refine > cfg->max_refine) { why = "init_refine out of range"; return AVS_EINVAL; }
    if (cfg->model != AVS_SHAKHOV && cfg->model != AVS_RYKOV) { why = "bad model"; return AVS_EINVAL; }
    if (cfg->model == AVS_RYKOV && !(cfg->Zrot >= 1.0)) { why = "Zrot must be at least 1"; return AVS_EINVAL; }
    if (m->Nc <= 0 || m->Nf <= 0 || m->nbc < 0) { why = "empty mesh"; return AVS_EINVAL; }
    if (!m->faceL || !m->faceR || !m->An || !m->rL || !m->rR || !m->vol || (m->nbc > 0 && !m->bc)) {
        why = "null mesh array";
        return AVS_EINVAL;
    }
    for (int b = 0; b < m->nbc; ++b) {
        const int t = (int)m->bc[b * 6];
        if (t != AVS_BC_WALL && t != AVS_BC_FARFIELD) { why = "bad boundary type"; return AVS_EINVAL; }
        if (!(m->bc[b * 6 + 5] > 0)) { why = "boundary temperature must be positive"; return AVS_EINVAL; }
    }
    std::vector<int> cnt(m->Nc, 0);
    for (int f = 0; f < m->Nf; ++f) {
        const int L = m->faceL[f], R = m->faceR[f];
        if (L < 0 || L >= m->Nc) { why = "faceL out of range"; return AVS_EINVAL; }
        if (R >= m->Nc || (R < 0 && -1 - R >= m->nbc)) { why = "faceR out of range"; return AVS_EINVAL; }
        if (R == L) { why = "face joins a cell to itself"; return AVS_EINVAL; }
        if (++cnt[L] > AVS_MAXS) { why = "more than 6 faces on a cell"; return AVS_EINVAL; }
        if (R >= 0 && ++cnt[R] > AVS_MAXS) { why = "more than 6 faces on a cell"; return AVS_EINVAL; }
    }
    for (int i = 0; i < m->Nc; ++i)
        if (!(m->vol[i] > 0)) { why = "non-positive cell volume"; return AVS_EINVAL; }
    return AVS_OK;
}

// Cell -> face slots in face order; least-squares weights (inverse-distance
// squared, R6) and limiter eps^2 = (K vol^(1/D))^3.
avs_status setup_mesh(avs_ctx* c, const avs_mesh* m)
{
    const int D = c->D, Nc = c->Nc, Nf = c->Nf;
    std::vector<int> slot((size_t)Nc * AVS_MAXS, -1), nbr((size_t)Nc * AVS_MAXS, -1);
    std::vector<unsigned char> ns(Nc, 0);
    for (int f = 0; f < Nf; ++f) {
        const int L = m->faceL[f], R = m->faceR[f];
        slot[(size_t)L * AVS_MAXS + ns[L]] = 2 * f;
        nbr[(size_t)L * AVS_MAXS + ns[L]] = R >= 0 ? R : -1;
        ns[L]++;
        if (R >= 0) {
            slot[(size_t)R * AVS_MAXS + ns[R]] = 2 * f + 1;
            nbr[(size_t)R * AVS_MAXS + ns[R]] = L;
            ns[R]++;
        }
    }
    c->max_ns = 0;
    for (int i = 0; i < Nc; ++i) c->max_ns = std::max(c->max_ns, (int)ns[i]);
    std::vector<double> cg((size_t)Nc * AVS_MAXS * D, 0.0), r((size_t)Nc * AVS_MAXS * D, 0.0), eps2(Nc);
    for (int i = 0; i < Nc; ++i) {
        double M[9] = {0}, dv[AVS_MAXS][3], n2[AVS_MAXS];
        for (int s = 0; s < ns[i]; ++s) {
            const int sl = slot[(size_t)i * AVS_MAXS + s];
            const int f = sl >> 1;
            const bool isR = sl & 1;
            const double* rs = (isR ? m->rR : m->rL) + (size_t)f * D;
            const double* ro = (isR ? m->rL : m->rR) + (size_t)f * D;
            for (int a = 0; a < D; ++a) r[((size_t)i * AVS_MAXS + s) * D + a] = rs[a];
            n2[s] = 0.0;
            if (nbr[(size_t)i * AVS_MAXS + s] < 0) continue;
            for (int a = 0; a < D; ++a) {
                dv[s][a] = rs[a] - ro[a];
                n2[s] += dv[s][a] * dv[s][a];
            }
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) M[a * D + b] += dv[s][a] * dv[s][b] / n2[s];
        }
        double tr = 0.0;
        for (int a = 0; a < D; ++a) tr += M[a * D + a];
        double Mi[9] = {0};
        bool ok = false;
        if (D == 2) {
            const double det = M[0] * M[3] - M[1] * M[2];
            if (det > 1e-12 * tr * tr) {
                ok = true;
                Mi[0] = M[3] / det; Mi[1] = -M[1] / det; Mi[2] = -M[2] / det; Mi[3] = M[0] / det;
            }
        } else {
            const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8],
                         c02 = M[3] * M[7] - M[4] * M[6];
            const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
            if (det > 1e-12 * tr * tr * tr) {
                ok = true;
                Mi[0] = c00 / det; Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det; Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
                Mi[3] = c01 / det; Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det; Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
                Mi[6] = c02 / det; Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det; Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
            }
        }
        if (ok) {
            for (int s = 0; s < ns[i]; ++s) {
                if (nbr[(size_t)i * AVS_MAXS + s] < 0) continue;
                for (int a = 0; a < D; ++a) {
                    double v = 0.0;
                    for (int b = 0; b < D; ++b) v += Mi[a * D + b] * dv[s][b];
                    cg[((size_t)i * AVS_MAXS + s) * D + a] = v / n2[s];
                }
            }
        }
        eps2[i] = pow(c->cfg.lim_K * pow(m->vol[i], 1.0 / D), 3.0);
    }
    auto tof = [](const double* p, size_t n) {
        std::vector<float> v(n);
        for (size_t k = 0; k < n; ++k) v[k] = (float)p[k];
        return v;
    };
    const size_t nfd = (size_t)Nf * D, ncs = (size_t)Nc * AVS_MAXS, ncsd = ncs * D;
    if (dalloc(&c->faceL, Nf) || dalloc(&c->faceR, Nf) || dalloc(&c->An_d, nfd) || dalloc(&c->rL_d, nfd) ||
        dalloc(&c->rR_d, nfd) || dalloc(&c->An_f, nfd) || dalloc(&c->rL_f, nfd) || dalloc(&c->rR_f, nfd) ||
        dalloc(&c->vol, Nc) || dalloc(&c->bc, (size_t)std::max(1, c->nbc) * 6) || dalloc(&c->slot, ncs) ||
        dalloc(&c->nslot, Nc) || dalloc(&c->nbr, ncs) || dalloc(&c->cg_d, ncsd) || dalloc(&c->r_d, ncsd) ||
        dalloc(&c->eps2_d, Nc) || dalloc(&c->cg_f, ncsd) || dalloc(&c->r_f, ncsd) || dalloc(&c->eps2_f, Nc) ||
        dalloc(&c->AFf, (size_t)Nf * c->NW) || dalloc(&c->forder, Nf) || dalloc(&c->cmom, (size_t)Nc * AVS_CMOM_MAX) ||
        dalloc((unsigned char**)&c->cpar, (size_t)Nc * AVS_CELLPAR_BYTES) || dalloc(&c->clist, Nc) ||
        dalloc(&c->imp_dW, (size_t)Nc * c->NW) || dalloc(&c->imp_rhs0, (size_t)Nc * c->NW) ||
        dalloc(&c->imp_diag, Nc) || dalloc(&c->imp_Wta, (size_t)Nc * c->NW) ||
        dalloc(&c->imp_co, ncs * AVS_IMPSLOT_BYTES) || dalloc(&c->imp_nint, Nc) || dalloc(&c->imp_bar, 1))
        return fail(c, AVS_ENOMEM, "mesh arrays");
    cudaStream_t s = c->stream;
    CK(up(c->faceL, std::vector<int>(m->faceL, m->faceL + Nf), s));
    CK(up(c->faceR, std::vector<int>(m->faceR, m->faceR + Nf), s));
    CK(up(c->An_d, std::vector<double>(m->An, m->An + nfd), s));
    CK(up(c->rL_d, std::vector<double>(m->rL, m->rL + nfd), s));
    CK(up(c->rR_d, std::vector<double>(m->rR, m->rR + nfd), s));
    CK(up(c->An_f, tof(m->An, nfd), s));
    CK(up(c->rL_f, tof(m->rL, nfd), s));
    CK(up(c->rR_f, tof(m->rR, nfd), s));
    CK(up(c->vol, std::vector<double>(m->vol, m->vol + Nc), s));
    if (c->nbc > 0) CK(up(c->bc, std::vector<double>(m->bc, m->bc + (size_t)c->nbc * 6), s));
    CK(up(c->slot, slot, s));
    CK(up(c->nslot, ns, s));
    CK(up(c->nbr, nbr, s));
    CK(up(c->cg_d, cg, s));
    CK(up(c->r_d, r, s));
    CK(up(c->eps2_d, eps2, s));
    CK(up(c->cg_f, tof(cg.data(), ncsd), s));
    CK(up(c->r_f, tof(r.data(), ncsd), s));
    CK(up(c->eps2_f, tof(eps2.data(), Nc), s));
    // faces in the order of their lower cell index, so that the face blocks in
    // flight together read the f and gradient rows of nearby cells (L2 reuse)
    std::vector<int> order(Nf);
    for (int f = 0; f < Nf; ++f) order[f] = f;
    auto low = [&](int f) { const int R = m->faceR[f]; return R >= 0 ? std::min(m->faceL[f], R) : m->faceL[f]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return low(a) < low(b); });
    CK(up(c->forder, order, s));
    // greedy colouring in cell order (smallest colour no face neighbour has):
    // cells of one colour share no face (implicit sweeps)
    {
        std::vector<int> col(Nc, -1);
        c->ncolor = 0;
        for (int i = 0; i < Nc; ++i) {
            unsigned used = 0;
            for (int q = 0; q < ns[i]; ++q) {
                const int j = nbr[(size_t)i * AVS_MAXS + q];
                if (j >= 0 && col[j] >= 0) used |= 1u << col[j];
            }
            int k = 0;
            while (used & (1u << k)) ++k;
            col[i] = k;
            c->ncolor = std::max(c->ncolor, k + 1);
        }
        c->cstart.assign(c->ncolor + 1, 0);
        for (int i = 0; i < Nc; ++i) c->cstart[col[i] + 1]++;
        for (int k = 0; k < c->ncolor; ++k) c->cstart[k + 1] += c->cstart[k];
        std::vector<int> pos(c->cstart.begin(), c->cstart.end() - 1), cl(Nc);
        for (int i = 0; i < Nc; ++i) cl[pos[col[i]]++] = i;
        CK(up(c->clist, cl, s));
        if (dalloc(&c->cstart_d, c->ncolor + 1)) return fail(c, AVS_ENOMEM, "colour offsets");
        CK(up(c->cstart_d, c->cstart, s));
    }
    CK(cudaStreamSynchronize(s));    // host vectors go out of scope
    return AVS_OK;
}

// Step-0 AVS (Sec. 3.5, steps 1-3): base forest, then adaptation on the two
// pseudo cells g^eq(W_inf) and g^eq(rho_inf, 0, T_inf), repeated until it
// stops changing (at most max(1, max_refine) passes).
avs_status initial_tree(avs_ctx* c)
{
    const int D = c->D;
    int nbase = 1;
    for (int d = 0; d < D; ++d) nbase *= c->cfg.base[d];
    std::vector<int> lev(nbase, 0), bas(nbase);
    std::vector<uint32_t> key(nbase, 0u);
    for (int b = 0; b < nbase; ++b) bas[b] = b;
    CK(up(c->level, lev, c->stream));
    CK(up(c->base, bas, c->stream));
    CK(up(c->key, key, c->stream));
    c->Nv = nbase;
    c->Nvp = round_up(nbase, 32);
    CK(launch_geom(c));
    const int NW = c->NW;
    double Wp[2][6] = {{0}}, Wc[2][6];
    for (int m = 0; m < D + 2; ++m) Wp[0][m] = Wp[1][m] = c->cfg.W_inf[m];
    for (int d = 0; d < D; ++d) Wp[1][1 + d] = 0.0;
    if (c->model == AVS_RYKOV) Wp[0][D + 2] = Wp[1][D + 2] = c->cfg.W_inf[D + 1];   // T_r = T_t
    std::vector<double> wpv, wcv;
    for (int j = 0; j < 2; ++j) {
        cons_host(D, Wp[j], c->cfg.R, Wc[j]);
        if (c->model == AVS_RYKOV) {
            // rho E_rot = rho R T_r (K = 2), added to the total energy
            Wc[j][D + 2] = Wp[j][0] * c->cfg.R * Wp[j][D + 2];
            Wc[j][D + 1] += Wc[j][D + 2];
        }
        for (int m = 0; m < NW; ++m) {
            wpv.push_back(Wp[j][m]);
            wcv.push_back(Wc[j][m]);
        }
    }
    if (!(Wp[0][0] > 0) || !(Wp[0][D + 1] > 0)) return fail(c, AVS_EINVAL, "W_inf must have rho, T > 0");
    double* Wp_d = c->pseudo_W;
    double* Wc_d = c->pseudo_W + 2 * NW;
    CK(up(Wp_d, wpv, c->stream));
    CK(up(Wc_d, wcv, c->stream));
    // step 2 of Sec. 3.5: uniform splits of every element before the adaptation
    for (int p = 0; p < c->cfg.init_refine; ++p) {
        int Nn, sp, mg;
        avs_status st = apply_marks(c, &Nn, &sp, &mg, 1);
        if (st != AVS_OK) return st;
        swap_tree(c, Nn);
        CK(launch_geom(c));
    }
    const int passes = std::max(1, c->cfg.max_refine);
    for (int p = 0; p < passes; ++p) {
        CK(launch_maxwell(c, Wp_d, 2, 0.0, 0, c->pseudo_f, 1, c->Nvp));
        CK(launch_criterion(c, c->pseudo_f, 1, 2, c->Nvp, Wc_d, nullptr, 0, 1));
        int Nn, sp, mg;
        avs_status st = apply_marks(c, &Nn, &sp, &mg, 0);
        if (st != AVS_OK) return st;
        swap_tree(c, Nn);
        CK(launch_geom(c));
        if (sp == 0 && mg == 0) break;
    }
    return AVS_OK;
}

}  // namespace

extern "C" {

avs_status avs_create(const avs_config* cfg, const avs_mesh* mesh, void* cuda_stream, avs_ctx** out)
{
    if (!out) return AVS_EINVAL;
    *out = nullptr;
    std::string why;
    avs_status st = validate(cfg, mesh, why);
    if (st != AVS_OK) {
        fprintf(stderr, "avs_create: %s\n", why.c_str());
        return st;
    }
    avs_ctx* c = new avs_ctx();
    c->cfg = *cfg;
    c->D = cfg->dim;
    c->model = cfg->model;
    c->NA = cfg->model == AVS_RYKOV ? (cfg->dim == 2 ? 3 : 2) : (cfg->dim == 2 ? 2 : 1);
    c->NW = cfg->dim + 2 + (cfg->model == AVS_RYKOV ? 1 : 0);
    c->Nc = mesh->Nc;
    c->Nf = mesh->Nf;
    c->nbc = mesh->nbc;
    c->mixed = cfg->precision == AVS_MIXED;
    c->stream = (cudaStream_t)cuda_stream;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            c->nsm = 0;
    }
    if (c->cfg.corr_iters == 0) c->cfg.corr_iters = 3;
    // Eq. (4)-(5) with rho = T = L_ref = 1
    c->mu_ref = 15.0 * sqrt(2.0 * AVS_PI * cfg->R) * cfg->Kn /
                (2.0 * (5.0 - 2.0 * cfg->omega) * (7.0 - 2.0 * cfg->omega));
    long long nbase = 1;
    for (int d = 0; d < c->D; ++d) {
        c->hb[d] = (cfg->vhi[d] - cfg->vlo[d]) / (double)cfg->base[d];
        nbase *= cfg->base[d];
    }
    c->s_norm = (double)nbase;
    c->zs.n = cfg->nzones;
    c->zs.outside = cfg->zone_outside_level;
    c->zs.maxr = cfg->max_refine;
    for (int z = 0; z < cfg->nzones; ++z) {
        c->zs.level[z] = cfg->zones[z].level;
        for (int d = 0; d < 3; ++d) c->zs.c[z][d] = d < c->D ? cfg->zones[z].c[d] : 0.0;
        c->zs.r2in[z] = cfg->zones[z].r_in * cfg->zones[z].r_in;
        c->zs.r2out[z] = cfg->zones[z].r_out * cfg->zones[z].r_out;
    }
    // node capacity of the tree arrays: all leaves at max_refine, bounded
    long long full = nbase << (c->D * cfg->max_refine);
    long long cap = std::min<long long>(full, 1 << 23);
    if (cfg->max_nodes > 0) cap = std::min<long long>(cap, cfg->max_nodes);
    cap = std::max<long long>(cap, nbase);
    c->cap = (int)cap;
    const int capp = round_up(c->cap, 32);
    const int NW = c->NW;
#define AL(p, n) \
    if (dalloc(&(p), (n)) != cudaSuccess) { st = fail(c, AVS_ENOMEM, "allocation of " #p); goto bad; }
    AL(c->level, capp); AL(c->base, capp); AL(c->key, capp);
    AL(c->level2, capp); AL(c->base2, capp); AL(c->key2, capp);
    AL(c->src, capp); AL(c->kind, capp); AL(c->emit, capp);
    AL(c->newidx, 2 * (size_t)capp); AL(c->d_count, 4);
    AL(c->xi_d, (size_t)capp * c->D); AL(c->w_d, capp);
    AL(c->xi_f, (size_t)capp * c->D); AL(c->w_f, capp); AL(c->xi_p, (size_t)capp * c->D);
    AL(c->M, capp); AL(c->Mkey, capp); AL(c->ncap, capp);
    AL(c->pseudo_f, 2 * (size_t)c->NA * capp); AL(c->pseudo_W, 4 * NW);
    AL(c->crit_cp, 5 * (size_t)std::max(c->Nc, 2)); AL(c->crit_cp32, 8 * (size_t)std::max(c->Nc, 2));
    AL(c->Mlo, capp); AL(c->Mhi, capp); AL(c->Mthr, 4 * (size_t)capp);
    AL(c->rmom, 13 * (size_t)std::max(c->Nc, 2));
    AL(c->W[0], (size_t)c->Nc * NW); AL(c->W[1], (size_t)c->Nc * NW);
    AL(c->Wf, (size_t)c->Nc * NW); AL(c->q, (size_t)c->Nc * c->D);
    AL(c->dev_err, 1); AL(c->dt_key, 1); AL(c->gap_d, 1);
#undef AL
    if (cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream) != cudaSuccess) {
        st = fail(c, AVS_ECUDA, "memset");
        goto bad;
    }
    st = setup_mesh(c, mesh);
    if (st != AVS_OK) goto bad;
    st = initial_tree(c);
    if (st != AVS_OK) goto bad;
    {
        // room for 25 % growth; avs_adapt reallocates beyond that unless max_nodes is set
        int fnodes = cfg->max_nodes > 0 ? cfg->max_nodes : std::min(c->cap, c->Nv + c->Nv / 4 + 32);
        fnodes = std::max(fnodes, c->Nv);
        c->fcap = round_up(fnodes, 32);
        st = alloc_f(c, c->fcap, &c->f[0], &c->f[1]);
        if (st != AVS_OK) goto bad;
    }
    if (cudaMemsetAsync(c->W[0], 0, sizeof(double) * c->Nc * NW, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->W[1], 0, sizeof(double) * c->Nc * NW, c->stream) != cudaSuccess) {
        st = fail(c, AVS_ECUDA, "memset");
        goto bad;
    }
    st = refresh_dt(c);
    if (st != AVS_OK) goto bad;
    *out = c;
    return AVS_OK;
bad:
    fprintf(stderr, "avs_create: %s\n", c->err.c_str());
    free_all(c);
    delete c;
    return st;
}

void avs_destroy(avs_ctx* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

const char* avs_last_error(const avs_ctx* c) { return c ? c->err.c_str() : "null context"; }
int avs_num_nodes(const avs_ctx* c) { return c ? c->Nv : 0; }
int avs_num_cells(const avs_ctx* c) { return c ? c->Nc : 0; }

avs_status avs_init_field(avs_ctx* c, const double* Wp, int is_device, double amp, uint64_t seed)
{
    if (!c || !Wp) return AVS_EINVAL;
    c->mom_valid = 0;                 // f or W change outside a step
    const size_t n = (size_t)c->Nc * c->NW;
    const double* Wp_d = Wp;
    if (!is_device) {
        CK(cudaMemcpyAsync(c->Wf, Wp, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        Wp_d = c->Wf;
    }
    CK(launch_maxwell(c, Wp_d, c->Nc, amp, seed, c->f[c->cur], 0, c->Nvp));
    if (c->model == AVS_SHAKHOV) {
        // W of the primitive input: the reference velocity of the moment sums below
        k_prim_to_cons<<<(c->Nc + 255) / 256, 256, 0, c->stream>>>(c->D, c->Nc, Wp_d, c->cfg.R, c->W[c->wcur]);
        c->launches += 1;
        CK(cudaGetLastError());
    }
    // carried W = moments of the discrete initial f (Eq. 7)
    CK(launch_cell_moments(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->W[c->wcur], nullptr));
    if (!is_device) CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_dt(avs_ctx* c, double cfl, double* dt_out)
{
    if (!c || !dt_out || !(cfl > 0)) return AVS_EINVAL;
    *dt_out = cfl * c->dt_unit;
    return AVS_OK;
}

avs_status ugks_step_dt(avs_ctx* c, int nsteps, double dt)
{
    if (!c || nsteps < 0 || !(dt > 0)) return AVS_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (c->model == AVS_RYKOV)
            CK(rk_launch_step(c, c->f[c->cur], c->f[c->cur ^ 1], c->W[c->wcur], c->W[c->wcur ^ 1], dt));
        else
            CK(launch_step(c, c->f[c->cur], c->f[c->cur ^ 1], c->W[c->wcur], c->W[c->wcur ^ 1], dt));
        c->cur ^= 1;
        c->wcur ^= 1;
    }
    return AVS_OK;
}

avs_status ugks_step_implicit(avs_ctx* c, int nsteps, double dt, int k_macro, int k_micro)
{
    if (!c || nsteps < 0 || !(dt > 0) || k_macro < 0 || k_micro < 0) return AVS_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (c->model == AVS_RYKOV)
            CK(rk_launch_step_implicit(c, c->f[c->cur], c->f[c->cur ^ 1], c->W[c->wcur], c->W[c->wcur ^ 1], dt,
                                       k_macro, k_micro));
        else
            CK(launch_step_implicit(c, c->f[c->cur], c->f[c->cur ^ 1], c->W[c->wcur], c->W[c->wcur ^ 1], dt, k_macro,
                                    k_micro));
        c->cur ^= 1;
        c->wcur ^= 1;
    }
    return AVS_OK;
}

// Adaptive parameters of Sec. 3.5 (domain, levels, zones, thresholds) from the flow data.
avs_status avs_paper_parameters(const avs_flow_spec* sp, avs_config* cfg)
{
    if (!sp || !cfg) return AVS_EINVAL;
    const int D = sp->dim;
    if (D != 2 && D != 3) return AVS_EINVAL;
    if (!(sp->Ma > 0) || !(sp->gamma > 1) || !(sp->R > 0) || !(sp->T_inf > 0) || !(sp->T_w > 0) ||
        !(sp->h_std > 0) || !(sp->rdv_sigma > 0))
        return AVS_EINVAL;
    double nd = 0.0;
    for (int d = 0; d < D; ++d) nd += sp->dir[d] * sp->dir[d];
    if (!(nd > 0) || !std::isfinite(nd)) return AVS_EINVAL;
    nd = sqrt(nd);
    const double sig_inf = sqrt(sp->R * sp->T_inf);
    const double T0 = sp->T_inf * (1.0 + 0.5 * (sp->gamma - 1.0) * sp->Ma * sp->Ma);
    const double sig0 = sqrt(sp->R * T0);
    const double sigw = sqrt(sp->R * sp->T_w);
    const double Uinf = sp->Ma * sqrt(sp->gamma * sp->R * sp->T_inf);
    double u[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; ++d) u[d] = Uinf * (sp->dir[d] / nd);
    const double Rdv = sp->rdv_sigma * sig0;
    const double ratio = 2.0 * Rdv / sp->h_std;
    int Lmax = 0;
    while (ldexp(1.0, Lmax) < ratio) {
        if (++Lmax > 30) return AVS_EINVAL;
    }
    const int Lw = (sp->T_w / sp->T_inf < 4.0) ? Lmax : Lmax - 1;
    const int Lmin = std::min((D == 2 && sp->Ma > 5.0) ? 4 : 3, Lmax);
    const int Lsep = std::max(Lmin, Lw - 1);
    if (D * Lmin > 24 || D * (Lmax - Lmin) > 30) return AVS_EINVAL;
    cfg->dim = D;
    for (int d = 0; d < 3; ++d) {
        const double c0 = d < D ? 0.4 * u[d] : 0.0;
        cfg->base[d] = d < D ? (1 << Lmin) : 1;
        cfg->vlo[d] = d < D ? c0 - Rdv : 0.0;
        cfg->vhi[d] = d < D ? c0 + Rdv : 0.0;
    }
    cfg->max_refine = Lmax - Lmin;
    cfg->zone_outside_level = 0;
    memset(cfg->zones, 0, sizeof(cfg->zones));
    for (int d = 0; d < D; ++d) cfg->zones[0].c[d] = u[d];
    cfg->zones[0].r_in = 0.0;
    cfg->zones[0].r_out = 3.0 * sig_inf;
    cfg->zones[0].level = Lmax - Lmin;
    cfg->zones[1].r_in = 0.0;
    cfg->zones[1].r_out = 3.0 * sigw;
    cfg->zones[1].level = std::max(0, Lw - Lmin);
    cfg->nzones = 2;
    if (sp->separated) {
        cfg->zones[2].r_in = 3.0 * sigw;
        cfg->zones[2].r_out = 5.0 * sigw;
        cfg->zones[2].level = Lsep - Lmin;
        cfg->nzones = 3;
    }
    cfg->init_refine = std::max(0, Lw - 1 - Lmin);
    cfg->C1 = 13.749 * pow(sp->Ma, -1.465);
    cfg->C2 = 3.3546e-4 * cfg->C1;
    return AVS_OK;
}

avs_status avs_grid_barrier_check(avs_ctx* c, int blocks, int rounds, int short_by, int* passed)
{
    if (!c || blocks <= 0 || rounds <= 0 || short_by < 0 || !passed) return AVS_EINVAL;
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (blocks > nsm) return fail(c, AVS_EINVAL, "grid barrier check: more blocks than SMs");
    int* d = nullptr;
    if (dalloc(&d, 1) != cudaSuccess) return fail(c, AVS_ENOMEM, "grid barrier check");
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_grid_barrier_check(c, blocks, rounds, short_by, d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(passed, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    CK(e);
    return read_err(c);
}

avs_status avs_stage_wait_check(avs_ctx* c, int arrive, int* completed)
{
    if (!c || !completed) return AVS_EINVAL;
    float src[32];
    for (int j = 0; j < 32; ++j) src[j] = 0.5f + (float)j;
    float* d = nullptr;
    int* dc = nullptr;
    if (dalloc(&d, 32) != cudaSuccess || dalloc(&dc, 1) != cudaSuccess) {
        cudaFree(d);
        return fail(c, AVS_ENOMEM, "staged-copy wait check");
    }
    cudaError_t e = cudaMemcpyAsync(d, src, sizeof(src), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_stage_wait_check(c, d, arrive != 0, dc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(completed, dc, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    cudaFree(dc);
    CK(e);
    return read_err(c);
}

avs_status ugks_step(avs_ctx* c, int nsteps, double cfl, double* dt_out)
{
    if (!c || !(cfl > 0)) return AVS_EINVAL;
    const double dt = cfl * c->dt_unit;
    if (dt_out) *dt_out = dt;
    return ugks_step_dt(c, nsteps, dt);
}

avs_status avs_adapt(avs_ctx* c, const avs_adapt_opts* opts, avs_adapt_stats* stats)
{
    if (!c) return AVS_EINVAL;
    c->mom_valid = 0;                 // f or W change outside a step
    avs_adapt_opts o = {};
    if (opts) o = *opts;
    const int NW = c->NW;
    const int Nv_old = c->Nv, Nvp_old = c->Nvp;
    // moments of f on the old mesh (Eq. 7): criterion input and correction
    // target; with the proposer also the heat flux of its features
    CK(launch_cell_moments(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, c->cfg.learned ? c->q : nullptr));
    if (o.W_override) {
        CK(cudaMemcpyAsync(c->Wf, o.W_override, sizeof(double) * c->Nc * NW,
                           o.W_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    }
    int checked = c->Nc, missed = 0, full = 1;
    c->mlp_checked_last = -1;
    if (c->cfg.learned) {
        avs_status s2 = ensure_mlp(c, c->Nc);
        if (s2 != AVS_OK) return s2;
        const int every = std::max(1, c->cfg.learned_full_every);
        full = o.force_full || c->mlp_trained == 0 || (c->adapt_count % every) == 0;
        // features of the current state: moments and heat flux of f
        CK(mlp_features(c, c->Wf, c->q, c->mlp_X));
        if (c->mlp_trained > 0) {
            // the proposer's check set and the criterion restricted to it
            CK(mlp_forward(c, c->Nc, c->mlp_X, c->mlp_logits));
            CK(mlp_checkset(c, c->mlp_logits, c->mlp_zthr, c->mlp_list, c->mlp_count));
            CK(cudaMemcpyAsync(&checked, c->mlp_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            c->mlp_checked_last = checked;
            CK(launch_criterion(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, c->mlp_list, checked, 1));
        }
        if (full) {
            if (c->mlp_trained > 0)
                CK(cudaMemcpyAsync(c->M_alt, c->M, sizeof(double) * c->Nv, cudaMemcpyDeviceToDevice, c->stream));
            // the plain criterion: fallback, judge of the misses and source of the labels
            // (exact M: the dominant label compares with it)
            CK(launch_criterion(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, nullptr, 0, 0));
            if (c->mlp_trained > 0) {
                CK(mlp_misses(c, c->M, c->M_alt, c->mlp_count + 1));
                CK(cudaMemcpyAsync(&missed, c->mlp_count + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
                CK(cudaStreamSynchronize(c->stream));
                // the full criterion judges the check set: widen it when it missed
                // more than 1 % of the nodes, narrow it when it missed none
                if (missed > c->Nv / 100) c->mlp_budget = std::min(1.0f, 2.0f * c->mlp_budget);
                else if (missed == 0) c->mlp_budget = std::max(0.05f, 0.8f * c->mlp_budget);
            }
            CK(mlp_labels(c, c->f[c->cur], c->mlp_Y));
            for (int it = 0; it < c->mlp_train_iters; ++it)
                CK(mlp_grad_step(c, c->Nc, c->mlp_X, c->mlp_Y, c->mlp_lr, c->mlp_grad));
            c->mlp_trained += c->mlp_train_iters;
            CK(mlp_calibrate(c, c->mlp_budget));
            checked = c->Nc;
        }
    } else {
        CK(launch_criterion(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, nullptr, 0, 1));
    }
    int Nn, sp, mg;
    avs_status st = apply_marks(c, &Nn, &sp, &mg, 0);
    if (st != AVS_OK) return st;
    const int Nvp_new = round_up(Nn, 32);
    void* dst = c->f[c->cur ^ 1];
    void *n0 = nullptr, *n1 = nullptr;
    if (Nvp_new > c->fcap) {
        if (c->cfg.max_nodes > 0) return fail(c, AVS_ECAPACITY, "adapted node count exceeds max_nodes");
        st = alloc_f(c, Nvp_new + Nvp_new / 2, &n0, &n1);
        if (st != AVS_OK) return st;
        dst = n0;
    }
    if (!o.bypass) CK(launch_remap(c, c->f[c->cur], Nvp_old, dst, Nvp_new, Nn));
    swap_tree(c, Nn);
    CK(launch_geom(c));
    if (o.bypass) {
        // f = g^eq(W) of the carried W on the new mesh (the bypass of Sec. 3.3)
        if (c->model == AVS_RYKOV) {
            CK(rk_launch_cons_to_prim(c, c->W[c->wcur], c->Wf));
        } else {
            k_cons_to_prim<<<(c->Nc + 255) / 256, 256, 0, c->stream>>>(c->D, c->Nc, c->W[c->wcur], c->cfg.R, c->Wf);
            c->launches += 1;
        }
        CK(launch_maxwell(c, c->Wf, c->Nc, 0.0, 0, dst, 0, Nvp_new));
    }
    if (n0) {
        CK(cudaStreamSynchronize(c->stream));
        cudaFree(c->f[0]);
        cudaFree(c->f[1]);
        c->f[0] = n0;
        c->f[1] = n1;
        c->fcap = round_up(Nvp_new + Nvp_new / 2, 32);
        c->cur = 0;
    } else {
        c->cur ^= 1;
    }
    double gap = 0.0;
    if (!o.skip_correction && !o.bypass) {
        CK(launch_correct(c, c->f[c->cur], c->Wf, c->cfg.corr_iters));
        unsigned long long gk = 0;
        CK(cudaMemcpyAsync(&gk, c->gap_d, sizeof(gk), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        gap = dkey_inv(gk);
    }
    st = refresh_dt(c);
    if (st != AVS_OK) return st;
    c->adapt_count++;
    if (stats) {
        stats->Nv_old = Nv_old;
        stats->Nv = c->Nv;
        stats->splits = sp;
        stats->merges = mg;
        stats->gap = gap;
        stats->checked_cells = checked;
        stats->missed_nodes = missed;
        stats->full = full;
    }
    (void)Nv_old;
    return read_err(c);
}

avs_status avs_moments(avs_ctx* c, double* Wc_out, double* q_out, int is_device)
{
    if (!c) return AVS_EINVAL;
    const cudaMemcpyKind kd = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (Wc_out)
        CK(cudaMemcpyAsync(Wc_out, c->W[c->wcur], sizeof(double) * c->Nc * c->NW, kd, c->stream));
    if (q_out) {
        CK(launch_cell_moments(c, c->f[c->cur], 0, c->Nc, c->Nvp, nullptr, c->q));
        CK(cudaMemcpyAsync(q_out, c->q, sizeof(double) * c->Nc * c->D, kd, c->stream));
    }
    if (!is_device) return read_err(c);
    return AVS_OK;
}

avs_status avs_f_moments(avs_ctx* c, double* Wc_out, int is_device)
{
    if (!c || !Wc_out) return AVS_EINVAL;
    CK(launch_cell_moments(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, nullptr));
    CK(cudaMemcpyAsync(Wc_out, c->Wf, sizeof(double) * c->Nc * c->NW,
                       is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!is_device) CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_set_W(avs_ctx* c, const double* Wc, int is_device)
{
    if (!c || !Wc) return AVS_EINVAL;
    c->mom_valid = 0;                 // f or W change outside a step
    CK(cudaMemcpyAsync(c->W[c->wcur], Wc, sizeof(double) * c->Nc * c->NW,
                       is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!is_device) CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_criterion(avs_ctx* c, const double* Wc, int W_is_device, double* M_out, int M_is_device)
{
    if (!c || !M_out) return AVS_EINVAL;
    const int NW = c->NW;
    if (Wc)
        CK(cudaMemcpyAsync(c->Wf, Wc, sizeof(double) * c->Nc * NW,
                           W_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    else
        CK(launch_cell_moments(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, nullptr));
    CK(launch_criterion(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, nullptr, 0, 0));
    CK(cudaMemcpyAsync(M_out, c->M, sizeof(double) * c->Nv,
                       M_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!M_is_device || !W_is_device) CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_get_tree(avs_ctx* c, int* level, int* base, uint32_t* key, double* xi, double* w)
{
    if (!c) return AVS_EINVAL;
    const size_t n = c->Nv;
    if (level) CK(cudaMemcpyAsync(level, c->level, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (base) CK(cudaMemcpyAsync(base, c->base, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (key) CK(cudaMemcpyAsync(key, c->key, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    if (xi) CK(cudaMemcpyAsync(xi, c->xi_d, n * c->D * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (w) CK(cudaMemcpyAsync(w, c->w_d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_get_f(avs_ctx* c, double* f, int is_device)
{
    if (!c || !f) return AVS_EINVAL;
    const size_t n = (size_t)c->Nc * c->NA * c->Nv;
    if (is_device) {
        CK(launch_to_double(c, c->f[c->cur], f, c->Nvp));
        return AVS_OK;
    }
    avs_status st = ensure_stage(c);
    if (st != AVS_OK) return st;
    CK(launch_to_double(c, c->f[c->cur], c->stage, c->Nvp));
    CK(cudaMemcpyAsync(f, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_get_f_cells(avs_ctx* c, const int* cells, int ncells, double* out)
{
    if (!c || !cells || !out || ncells < 0) return AVS_EINVAL;
    for (int j = 0; j < ncells; ++j)
        if (cells[j] < 0 || cells[j] >= c->Nc) return fail(c, AVS_EINVAL, "cell index out of range");
    if (ncells == 0) return AVS_OK;
    const size_t n = (size_t)ncells * c->NA * c->Nv;
    int* cells_d = nullptr;
    double* buf = nullptr;
    if (cudaMalloc(&cells_d, sizeof(int) * ncells) != cudaSuccess) return fail(c, AVS_ENOMEM, "cell list");
    if (cudaMalloc(&buf, sizeof(double) * n) != cudaSuccess) {
        cudaFree(cells_d);
        return fail(c, AVS_ENOMEM, "gather buffer");
    }
    cudaError_t e = cudaMemcpyAsync(cells_d, cells, sizeof(int) * ncells, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_gather_double(c, cells_d, ncells, buf);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(cells_d);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(c, AVS_ECUDA, cudaGetErrorString(e));
    return read_err(c);
}

avs_status avs_set_f(avs_ctx* c, const double* f, int is_device)
{
    if (!c || !f) return AVS_EINVAL;
    c->mom_valid = 0;                 // f or W change outside a step
    const size_t n = (size_t)c->Nc * c->NA * c->Nv;
    if (is_device) {
        CK(launch_from_double(c, f, c->f[c->cur], c->Nvp));
        return AVS_OK;
    }
    avs_status st = ensure_stage(c);
    if (st != AVS_OK) return st;
    CK(cudaMemcpyAsync(c->stage, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(launch_from_double(c, c->stage, c->f[c->cur], c->Nvp));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

uint64_t avs_kernel_launches(const avs_ctx* c) { return c ? (uint64_t)c->launches : 0; }

avs_status avs_mlp_set_params(avs_ctx* c, const float* params)
{
    if (!c || !params) return AVS_EINVAL;
    avs_status st = ensure_mlp(c, c->Nc);
    if (st != AVS_OK) return st;
    CK(cudaMemcpyAsync(c->mlp_P, params, sizeof(float) * AVS_MLP_NPARAM, cudaMemcpyHostToDevice, c->stream));
    CK(mlp_prep(c));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_mlp_get_params(avs_ctx* c, float* params)
{
    if (!c || !params) return AVS_EINVAL;
    avs_status st = ensure_mlp(c, c->Nc);
    if (st != AVS_OK) return st;
    CK(cudaMemcpyAsync(params, c->mlp_P, sizeof(float) * AVS_MLP_NPARAM, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_mlp_forward(avs_ctx* c, const float* X, int n, float* logits)
{
    if (!c || !X || !logits || n < 0) return AVS_EINVAL;
    avs_status st = ensure_mlp(c, n);
    if (st != AVS_OK) return st;
    CK(cudaMemcpyAsync(c->mlp_X, X, sizeof(float) * 8 * n, cudaMemcpyHostToDevice, c->stream));
    CK(mlp_forward(c, n, c->mlp_X, c->mlp_logits));
    CK(cudaMemcpyAsync(logits, c->mlp_logits, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_mlp_grad(avs_ctx* c, const float* X, const float* Y, int n, float lr, float* grad_out, float* loss_out)
{
    if (!c || !X || !Y || n <= 0) return AVS_EINVAL;
    avs_status st = ensure_mlp(c, n);
    if (st != AVS_OK) return st;
    CK(cudaMemcpyAsync(c->mlp_X, X, sizeof(float) * 8 * n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->mlp_Y, Y, sizeof(float) * 4 * n, cudaMemcpyHostToDevice, c->stream));
    CK(mlp_grad_step(c, n, c->mlp_X, c->mlp_Y, lr, c->mlp_grad));
    std::vector<float> g(AVS_MLP_NPARAM + 1);
    CK(cudaMemcpyAsync(g.data(), c->mlp_grad, sizeof(float) * g.size(), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (grad_out) memcpy(grad_out, g.data(), sizeof(float) * AVS_MLP_NPARAM);
    if (loss_out) *loss_out = g[AVS_MLP_NPARAM];
    return AVS_OK;
}

avs_status avs_features(avs_ctx* c, float* X_out, float* Y_out)
{
    if (!c) return AVS_EINVAL;
    avs_status st = ensure_mlp(c, c->Nc);
    if (st != AVS_OK) return st;
    CK(launch_cell_moments(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, c->q));
    CK(mlp_features(c, c->Wf, c->q, c->mlp_X));
    CK(launch_criterion(c, c->f[c->cur], 0, c->Nc, c->Nvp, c->Wf, nullptr, 0, 0));
    CK(mlp_labels(c, c->f[c->cur], c->mlp_Y));
    if (X_out) CK(cudaMemcpyAsync(X_out, c->mlp_X, sizeof(float) * 8 * c->Nc, cudaMemcpyDeviceToHost, c->stream));
    if (Y_out) CK(cudaMemcpyAsync(Y_out, c->mlp_Y, sizeof(float) * 4 * c->Nc, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return AVS_OK;
}

avs_status avs_mlp_train(avs_ctx* c, int iters, float lr, float* loss_out)
{
    if (!c || iters < 0) return AVS_EINVAL;
    avs_status st = avs_features(c, nullptr, nullptr);
    if (st != AVS_OK) return st;
    for (int it = 0; it < iters; ++it) CK(mlp_grad_step(c, c->Nc, c->mlp_X, c->mlp_Y, lr, c->mlp_grad));
    c->mlp_trained += iters;
    if (iters > 0) CK(mlp_calibrate(c, c->mlp_budget));
    if (loss_out) {
        float g = 0.f;
        CK(cudaMemcpyAsync(&g, c->mlp_grad + AVS_MLP_NPARAM, sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *loss_out = g;
    }
    return AVS_OK;
}

avs_status avs_mlp_check_set(avs_ctx* c, int* cells_out, int* n_out)
{
    if (!c || !n_out) return AVS_EINVAL;
    *n_out = c->mlp_checked_last;
    if (c->mlp_checked_last > 0 && cells_out) {
        CK(cudaMemcpyAsync(cells_out, c->mlp_list, sizeof(int) * c->mlp_checked_last, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return AVS_OK;
}

avs_status avs_sync(avs_ctx* c)
{
    if (!c) return AVS_EINVAL;
    return read_err(c);
}

}  // extern "C"
