// Host-side context of the AVS/UGKS library and the launchers shared by the
// translation units.  Not part of the public ABI (see include/avs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/avs.h"

#define AVS_NT 256            // threads per block of the per-cell kernels
#define AVS_CELLPAR_BYTES 256 // bytes per cell of the collision parameters (CellPar)
#define AVS_CMOM_MAX 17       // carried raw moments per cell (monatomic 11 / 13, Rykov 14 / 17)
#define AVS_SMALL_ROW_BYTES 8192 // f rows of a cell up to this size: one warp per face in the mixed step
#define AVS_IMPSLOT_BYTES 96  // bytes per slot record of the implicit macroscopic sweep

// Refinement caps of the velocity nodes (Sec. 3.5), passed to kernels by value.
struct ZoneSet {
    int n = 0;               // zones in use; 0: every node may split up to maxr
    int outside = 0;         // cap of a node in no zone
    int maxr = 0;            // max_refine
    int level[AVS_MAX_ZONES] = {0, 0, 0, 0};
    double c[AVS_MAX_ZONES][3] = {};
    double r2in[AVS_MAX_ZONES] = {}, r2out[AVS_MAX_ZONES] = {};
};

struct avs_ctx {
    avs_config cfg;
    ZoneSet zs;
    int D = 2, NA = 2, Nc = 0, Nf = 0, nbc = 0;
    int model = 0;           // AVS_SHAKHOV or AVS_RYKOV
    int NW = 4;              // conserved variables per cell: D+2, or D+3 for the Rykov model
    int mixed = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    double mu_ref = 0.0;     // from Kn, Eq. (5)
    double hb[3] = {0, 0, 0};
    double s_norm = 1.0;     // number of base-forest nodes
    int adapt_count = 0;

    // ---- physical mesh (device)
    int *faceL = nullptr, *faceR = nullptr;          // [Nf]
    double *An_d = nullptr, *rL_d = nullptr, *rR_d = nullptr;  // [Nf][D]
    float *An_f = nullptr, *rL_f = nullptr, *rR_f = nullptr;
    double *vol = nullptr;                           // [Nc]
    double *bc = nullptr;                            // [nbc][6]
    int *slot = nullptr;                             // [Nc][MAXS] face*2 + (cell is R), -1 none
    unsigned char *nslot = nullptr;                  // [Nc]
    int max_ns = 0;                                  // largest face count of a cell
    int *nbr = nullptr;                              // [Nc][MAXS]
    double *cg_d = nullptr, *r_d = nullptr, *eps2_d = nullptr;
    float *cg_f = nullptr, *r_f = nullptr, *eps2_f = nullptr;

    // ---- velocity tree (device), capacity `cap` nodes
    int Nv = 0, Nvp = 0, cap = 0;
    int *level = nullptr, *base = nullptr;
    uint32_t *key = nullptr;
    int *level2 = nullptr, *base2 = nullptr;
    uint32_t *key2 = nullptr;
    int *src = nullptr, *kind = nullptr, *emit = nullptr, *newidx = nullptr;
    int *d_count = nullptr;
    double *xi_d = nullptr, *w_d = nullptr;          // [cap][D], [cap]
    int *ncap = nullptr;                             // [cap] largest level a node may split to (zones)
    float *xi_f = nullptr, *w_f = nullptr;
    float *xi_p = nullptr;                           // FP32 node coordinates by pairs: [cap/2][D][2]
    double *M = nullptr;                             // [cap]
    unsigned long long *Mkey = nullptr;              // [cap]

    // ---- state (device)
    void *f[2] = {nullptr, nullptr};                 // [Nc][NA][Nvp] of T, capacity fcap nodes
    int fcap = 0;                                    // node capacity of the f buffers
    int cur = 0;
    double *W[2] = {nullptr, nullptr};               // carried conserved W, [Nc][D+2]
    int wcur = 0;
    double *Wf = nullptr;                            // moments of f / correction target
    double *q = nullptr;                             // [Nc][D]
    double *pseudo_f = nullptr;                      // step-0 pseudo cells [2][NA][cap]
    double *pseudo_W = nullptr;                      // [2][D+2]
    double *crit_cp = nullptr;                       // criterion per-cell inputs [max(Nc,2)][5]
    float *crit_cp32 = nullptr;                      // their FP32 screening form [max(Nc,2)][8]
    unsigned *Mlo = nullptr;                         // [cap] screening lower bounds of M (ordered keys)
    unsigned *Mhi = nullptr;                         // [cap] screening upper bounds of M
    float *Mthr = nullptr;                           // [cap][4] label thresholds per node
    double *stage = nullptr;                         // FP64 staging [Nc][NA][Nv] for get/set (lazy)
    size_t stage_elems = 0;
    int *dev_err = nullptr;                          // device error word (1: numeric, 2: grid barrier, 4: staged copy)
    unsigned long long *dt_key = nullptr;
    double *gap_d = nullptr;                         // correction gap (max over cells)
    double dt_unit = 0.0;
    unsigned long long launches = 0;                 // kernels launched by this context
    void *grad = nullptr;                            // limited gradients [Nc][NA][D][Nvp] of T
    size_t grad_bytes = 0;
    void *flux = nullptr;                            // per-node face flux [Nf][NA][Nvp] of T
    size_t flux_bytes = 0;
    double *AFf = nullptr;                           // area-weighted face flux of W [Nf][D+2]
    int *forder = nullptr;                           // face processing order (by lower cell index)
    double *cmom = nullptr;                          // raw moments of f about U(W) per cell [Nc][NMom]
    double *rmom = nullptr;                          // scratch raw moments [max(Nc,2)][NMom]
    int mom_valid = 0;                               // cmom matches the current f and W
    void *cpar = nullptr;                            // per-cell collision parameters (k_cell_state)

    // ---- implicit step (Sec. 2.3.1): cell colouring and the macroscopic system
    int ncolor = 0;
    std::vector<int> cstart;                         // [ncolor+1] offsets into clist (host)
    int *clist = nullptr;                            // [Nc] cells by colour, ascending within a colour
    int *cstart_d = nullptr;                         // [ncolor+1] the same offsets on the device
    double *imp_dW = nullptr, *imp_rhs0 = nullptr;   // [Nc][NW] (dW and -sum sgn A F, in the sweep type)
    double *imp_Wta = nullptr;                       // [Nc][NW] W~ in FP32 (mixed form)
    double *imp_diag = nullptr;                      // [Nc]
    unsigned char *imp_co = nullptr;                 // [Nc][MAXS] interior slot records (AVS_IMPSLOT_BYTES each)
    unsigned char *imp_nint = nullptr;               // [Nc] interior slots per cell in sweep order
    unsigned *imp_bar = nullptr;                     // grid barrier counter of the macroscopic solve
    int nsm = 0;                                     // multiprocessors of the device

    // ---- learned proposer (MLP 8-64-64-4)
    float *mlp_P = nullptr;                          // FP32 master parameters
    void *mlp_Wb = nullptr;                          // BF16 operand copies
    float *mlp_part = nullptr;                       // per-block gradient partials
    float *mlp_grad = nullptr;                       // gradient (+ loss) of the last step
    float *mlp_X = nullptr, *mlp_Y = nullptr;        // features / labels [Nc][8], [Nc][4]
    float *mlp_logits = nullptr;                     // [Nc][4]
    int *mlp_list = nullptr, *mlp_count = nullptr;   // check set
    int mlp_rows = 0;                                // row capacity of the MLP buffers
    double *M_alt = nullptr;                         // criterion over the check set
    int mlp_trained = 0;                             // training steps so far
    float mlp_lr = 0.1f;
    int mlp_train_iters = 50;
    float mlp_zthr = -1.0f;                          // logit threshold of the check set
    float mlp_budget = 0.25f;                        // fraction of cells in the check set
    int mlp_checked_last = -1;                       // size of the last adaptation's check set, -1 none
};

namespace avs {

int round_up(int n, int m);

// ---- launchers (avs_step.cu)
cudaError_t launch_step(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt);
// Rykov model (csrc/avs_rykov.cu)
// limited gradients of the Rykov arrays (3 in 2D, 2 in 3D) into c->grad
void launch_grad_rykov(avs_ctx* c, const void* fin);
cudaError_t rk_launch_step(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt);
cudaError_t rk_launch_step_implicit(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout,
                                    double dt, int k_macro, int k_micro);
cudaError_t rk_launch_moments(avs_ctx* c, const void* f, int f_is_double, int Ncells, int Nvp, double* Wout,
                              double* qout);
cudaError_t rk_launch_correct(avs_ctx* c, void* f, const double* Wtarget, int iters);
cudaError_t rk_launch_cons_to_prim(avs_ctx* c, const double* Wc, double* Wp);
cudaError_t launch_grid_barrier_check(avs_ctx* c, int blocks, int rounds, int short_by, int* passed_dev);
cudaError_t launch_stage_wait_check(avs_ctx* c, const float* src, bool arrive, int* completed_dev);
cudaError_t launch_step_implicit(avs_ctx* c, const void* fin, void* fout, const double* Win, double* Wout, double dt,
                                 int k_macro, int k_micro);

// ---- launchers (avs_adapt.cu)
cudaError_t launch_geom(avs_ctx* c);                       // xi, w of the current tree
cudaError_t launch_dt_unit(avs_ctx* c);                    // min |V|/sum max(xi.n,0) -> c->dt_key
cudaError_t launch_maxwell(avs_ctx* c, const double* Wp, int Ncells, double amp, uint64_t seed,
                           void* fout, int f_is_double, int Nvp);
cudaError_t launch_cell_moments(avs_ctx* c, const void* f, int f_is_double, int Ncells, int Nvp,
                                double* Wc_out, double* q_out);
cudaError_t launch_criterion(avs_ctx* c, const void* f, int f_is_double, int Ncells, int Nvp,
                             const double* Wc, const int* cells, int ncells_list, int decide);
// decide = 1: M exact only where the split/merge tests need it (marks); 0: M exact everywhere
cudaError_t launch_adapt_tree(avs_ctx* c, double C1, double C2, int uniform);  // marks, scan, new tree -> *2 arrays
cudaError_t launch_remap(avs_ctx* c, const void* fold, int Nvp_old, void* fnew, int Nvp_new, int Nv_new);
cudaError_t launch_correct(avs_ctx* c, void* f, const double* Wtarget, int iters);
cudaError_t launch_to_double(avs_ctx* c, const void* f, double* out, int Nvp);   // packed [Nc][NA][Nv]
cudaError_t launch_from_double(avs_ctx* c, const double* in, void* f, int Nvp);
cudaError_t launch_gather_double(avs_ctx* c, const int* cells_d, int ncells, double* out);   // [n][NA][Nv]

}  // namespace avs
