/*
 * avs.h — C ABI of the GB300 (sm_103a) library for the unified gas-kinetic
 * scheme (UGKS) on one global adaptive velocity space (AVS), following
 * Chen, Liu, Zhang, Zhong, Yang, Zhuo, arXiv 2212.05645.
 *
 * One context owns one problem on one GPU: the physical mesh, the global
 * quadtree/octree velocity mesh, the reduced distributions f (G and H in 2D,
 * G in 3D; Eq. 6) and the carried conserved variables W (Eq. 7).  Every call
 * enqueues its work on the context's CUDA stream.  Calls return an
 * avs_status and never throw; on error avs_last_error() describes it.  After
 * AVS_ECUDA the context must be destroyed; after any other error it stays
 * valid.  A context is not thread-safe.
 *
 * Pointers marked "host or device" are read or written on the host when the
 * accompanying is_device flag is 0 and on the device (same device as the
 * context, ordered on its stream) when it is 1.  Input pointers are borrowed
 * for the duration of the call only.  Output buffers are owned by the caller.
 *
 * Layouts (NW = D+2 for the Shakhov model, D+3 for the Rykov model)
 *   f    [cell][array][node]  (array 0 = G, array 1 = H in 2D; Rykov: last array R),
 *                             FP64 on the ABI
 *   Wc   [cell][NW]           conserved: rho, rho*U (D), rho*E (Rykov: total, with the
 *                             rotational energy), and for Rykov rho*E_rot
 *   Wp   [cell][NW]           primitive: rho, U (D), T (Rykov: T_t, T_r)
 *   q    [cell][D]            heat flux (Eq. 8)
 *   xi   [node][D], w [node]  velocity node (element centre) and weight (Sec. 3)
 */
#ifndef AVS_H
#define AVS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct avs_ctx avs_ctx;

typedef enum {
    AVS_OK = 0,
    AVS_EINVAL = -1,      /* bad argument, configuration or mesh           */
    AVS_ENOMEM = -2,      /* device or host allocation failed              */
    AVS_ECUDA = -3,       /* CUDA runtime error; the context is unusable   */
    AVS_ETIMEOUT = -4,    /* a bounded device wait gave up                 */
    AVS_ENUMERIC = -5,    /* non-positive density or temperature met       */
    AVS_ENOTCONV = -6,    /* conservation correction gap grew              */
    AVS_ECAPACITY = -7    /* adapted velocity mesh exceeds max_nodes, or a
                             problem beyond the fixed scratch of
                             avs_criterion_noalloc                          */
} avs_status;

enum { AVS_FP64 = 0, AVS_MIXED = 1 };
enum { AVS_SHAKHOV = 0, AVS_RYKOV = 1 };

/* Rykov coefficients for nitrogen (Sec. 2.1, after Eq. 13) */
#define AVS_RYKOV_DELTA (1.0 / 1.55)
#define AVS_RYKOV_OMEGA0 0.2354
#define AVS_RYKOV_OMEGA1 0.3049
enum { AVS_BC_WALL = 1, AVS_BC_FARFIELD = 2 };
enum { AVS_LIM_FIRST_ORDER = 0, AVS_LIM_VENKAT = 1, AVS_LIM_NONE = 2 };

#define AVS_MAX_ZONES 4

/* A refinement zone of the velocity space (Sec. 3.5): a node whose centre xi
 * has r_in^2 <= |xi - c|^2 < r_out^2 (FP64, no fused multiply-add) may be
 * split up to `level`, counted in levels above the base forest. */
typedef struct {
    double c[3];
    double r_in, r_out;
    int level;
} avs_zone;

/* Run configuration.  Units: rho_inf = T_inf = L_ref = 1 and velocity unit
 * sqrt(2 R T_inf), so R = 1/2 (paper Sec. 4.5 tables). */
typedef struct {
    int dim;              /* 2 or 3 (physical = velocity dimension)                        */
    int base[3];          /* base-forest elements per velocity axis (level 0, Sec. 3.5 step 2) */
    int max_refine;       /* largest tree level                                             */
    double vlo[3], vhi[3];/* velocity domain                                                */
    int precision;        /* AVS_FP64: f and all arithmetic in FP64.
                             AVS_MIXED: f, reconstruction, flux and collision in FP32;
                             moment sums, wall balance and correction in FP64              */
    int learned;          /* 1: the MLP proposer restricts the criterion to a check set      */
    double R, Pr, omega;  /* gas constant, Prandtl number (2/3), VHS exponent (Eq. 3)       */
    double Kn;            /* Knudsen number of the reference state (Eq. 5)                  */
    double T_ref;         /* reference temperature of the viscosity law                    */
    double C1, C2;        /* split / merge thresholds (Sec. 3.4) on s*M_k, s = base nodes   */
    double W_inf[5];      /* primitive free stream rho, U (dim), T for the step-0 AVS        */
    int limiter;          /* AVS_LIM_*; Venkatakrishnan with eps^2 = (lim_K dx)^3           */
    double lim_K;
    int corr_iters;       /* passes of the conservation correction (Sec. 3.3)               */
    int max_nodes;        /* velocity-node capacity (fixed); 0 = 1.25x the step-0 count, grown on demand */
    int learned_full_every; /* learned form: run the full criterion every n-th adaptation   */
    int nzones;           /* 0: any node may split up to max_refine.  1..AVS_MAX_ZONES: a node
                             may split up to the largest level of the zones holding its centre,
                             else up to zone_outside_level (Sec. 3.5)                        */
    int zone_outside_level;
    avs_zone zones[AVS_MAX_ZONES];
    int init_refine;      /* uniform splits of every base element before the step-0 adaptation
                             (Sec. 3.5 step 2); 0..max_refine                                */
    int model;            /* AVS_SHAKHOV (monatomic, Eqs. 14-17) or AVS_RYKOV (diatomic,
                             Eqs. GHR_equ, 11-13).  Rykov: f has the arrays G, H, R in 2D and
                             G, R in 3D; W adds rho E_rot (NW = D+3 values per cell); the
                             proposer's temperature features are those of T_t           */
    double Zrot;          /* rotational collision number Z_rot of the Rykov model (>= 1)     */
} avs_config;

/* Flow data for the adaptive parameters of Sec. 3.5 (avs_paper_parameters). */
typedef struct {
    int dim;              /* 2 or 3                                                          */
    double Ma;            /* free-stream Mach number |U_inf| / sqrt(gamma R T_inf)           */
    double gamma, R;      /* specific-heat ratio, gas constant (1/2 in these units)          */
    double T_inf, T_w;    /* free-stream static and wall temperature                         */
    double dir[3];        /* direction of U_inf (any length > 0)                             */
    double h_std;         /* standard velocity interval (0.6 in the paper)                   */
    double rdv_sigma;     /* R_dv / sigma_0: 4, or up to 7 when T_w is close to T_0          */
    int separated;        /* 1: add the separated zone 3 sigma_w < |xi| < 5 sigma_w          */
} avs_flow_spec;

/* Physical mesh as a face list (finite-volume form of Eq. 18).
 * faceR[f] < 0 marks a boundary face with condition -1 - faceR[f]; for those
 * faceL[f] is the interior cell and An points out of the domain.
 * bc[b*6 .. b*6+5] = type (AVS_BC_*), rho, U0, U1, U2, T: a wall uses U, T
 * (diffuse reflection, density from zero net mass flux); a far field imposes
 * the Maxwellian of (rho, U, T) on incoming velocities.  All host pointers. */
typedef struct {
    int dim, Nc, Nf, nbc;
    const int *faceL, *faceR;     /* [Nf]                                   */
    const double *An;             /* [Nf][dim] area * unit normal, L -> R   */
    const double *rL, *rR;        /* [Nf][dim] face centre - cell centre    */
    const double *vol;            /* [Nc]                                   */
    const double *bc;             /* [nbc][6]                               */
} avs_mesh;

typedef struct {
    int Nv_old, Nv, splits, merges;
    double gap;           /* largest relative |M[f] - W| after the correction */
    int checked_cells;    /* cells on which the criterion ran                 */
    int missed_nodes;     /* learned form: decisions the check set got wrong (full steps only) */
    int full;             /* 1 if the full criterion ran                      */
} avs_adapt_stats;

typedef struct {
    const double *W_override; /* nullable: conserved W [Nc][NW] used by the criterion and as
                                 the correction target instead of the moments of f           */
    int W_is_device;
    int skip_correction;      /* 1: remap only (Sec. 3.2), no Sec. 3.3 correction             */
    int force_full;           /* learned form: run the full criterion on this call            */
    int bypass;               /* 1: f on the new mesh is g^eq of the carried W (Sec. 3.3, the
                                 bypass for weakly non-equilibrium flows) instead of the remap
                                 and correction                                              */
} avs_adapt_opts;

/* Creates a context, uploads the mesh, builds the step-0 velocity mesh
 * (Sec. 3.5 steps 1-3: base forest, then adaptation on g^eq(W_inf) and
 * g^eq(rho_inf, 0, T_inf) repeated until it stops changing, at most
 * max_refine passes) and allocates f.  cuda_stream: cudaStream_t or NULL
 * for the default stream.  Errors: EINVAL (config/mesh), ENOMEM, ECUDA. */
avs_status avs_create(const avs_config *cfg, const avs_mesh *mesh, void *cuda_stream, avs_ctx **out);
void       avs_destroy(avs_ctx *ctx);
const char *avs_last_error(const avs_ctx *ctx);
int        avs_num_nodes(const avs_ctx *ctx);
int        avs_num_cells(const avs_ctx *ctx);

/* f = g^eq(Wp_i)(xi_k) (1 + amp z_ik), H = (3-D) R T G (Eq. 16), with z_ik a
 * standard normal from SplitMix64 (key (i << 32) | k, Box-Muller); then the
 * carried W = moments of f (Eq. 7).  Wp: primitive [Nc][NW], host or device.
 * Rykov model: G = g^eq(rho, U, T_t)(1 + amp z), H = (3-D) R T_t G,
 * R = R T_r G from Wp = (rho, U, T_t, T_r), and W by Eq. (updat_W). */
avs_status avs_init_field(avs_ctx *ctx, const double *Wp, int is_device, double amp, uint64_t seed);

/* dt = cfl * min over cells i and nodes k of |V_i| / sum_j A_ij max(xi_k . n_ij, 0). */
avs_status avs_dt(avs_ctx *ctx, double cfl, double *dt_out);

/* nsteps explicit UGKS steps (Sec. 2.3 with zero SGS sweeps): foot
 * reconstruction, interface moments and Shakhov state, simplified
 * multiscale flux (Eq. equ28), conservative W update, implicit-collision
 * update of f (diagonal of Eq. SGS_phi).  dt from cfl (avs_dt); dt_out
 * nullable.  Does not synchronise; numeric failures surface at the next
 * blocking call as AVS_ENUMERIC, and an asynchronous copy of the FP32 face
 * kernel that did not complete within its bound (about a second) as
 * AVS_ETIMEOUT. */
avs_status ugks_step(avs_ctx *ctx, int nsteps, double cfl, double *dt_out);
avs_status ugks_step_dt(avs_ctx *ctx, int nsteps, double dt);

/* nsteps implicit steps of size dt (IUGKS, Sec. 2.3.1): the interface
 * distribution and fluxes at t^n as in ugks_step, then the macroscopic
 * Eq. (SGS_w) for W~ - W^n (Roe-type flux differences; r = |U.n| + a +
 * 2 mu / (rho dl) from the mean state of the two cells) and the microscopic
 * Eq. (SGS_phi) for phi^{n+1} - phi^n, each solved by k_macro / k_micro
 * symmetric Gauss-Seidel iterations (a forward and a backward sweep over a
 * greedy cell colouring).  Boundary faces enter both diagonals with a fixed
 * ghost state.  Rykov model: the diatomic Euler flux (p from the equilibrium
 * temperature, rho E_rot carried) and radius (a = sqrt(7/5 R T)), and Eq.
 * (SGS_wrot) for rho E_rot with the rotational source taken from the cell's
 * current W~ and its implicit part in the diagonal.  The paper recommends
 * k_macro = 60, k_micro = 2.  The
 * macroscopic solve is one cooperative launch with a bounded grid barrier
 * between colour passes.  Does not synchronise.  Errors: EINVAL (nsteps < 0,
 * dt <= 0, negative sweep counts), ECUDA; at the next blocking call ENUMERIC
 * or ETIMEOUT (a grid barrier gave up). */
avs_status ugks_step_implicit(avs_ctx *ctx, int nsteps, double dt, int k_macro, int k_micro);

/* One AVS adaptation (Sec. 3): moments of f (Eq. 7), criterion M_k
 * (Eqs. criterion_rho/_e/_mk), split/merge marks, new depth-first tree,
 * consanguinity remap (Sec. 3.2), conservation correction (Sec. 3.3).
 * Blocks until the new node count is known.  opts and stats nullable.
 * Errors: ECAPACITY (tree would exceed max_nodes; state unchanged), ENUMERIC. */
avs_status avs_adapt(avs_ctx *ctx, const avs_adapt_opts *opts, avs_adapt_stats *stats);

/* Carried conserved W (FP64) and heat flux q of f (Eq. 8), host or device.
 * Either output may be NULL.  Blocks when writing to the host. */
avs_status avs_moments(avs_ctx *ctx, double *Wc_out, double *q_out, int is_device);
/* Conserved moments of f itself (Eq. 7). */
avs_status avs_f_moments(avs_ctx *ctx, double *Wc_out, int is_device);
avs_status avs_set_W(avs_ctx *ctx, const double *Wc, int is_device);

/* Criterion values M_k (unscaled) for the current f; Wc nullable (NULL: the
 * moments of f).  M_out: [Nv] host or device. */
avs_status avs_criterion(avs_ctx *ctx, const double *Wc, int W_is_device, double *M_out, int M_is_device);

/* Tree copy-out (host): level, base index, path key, xi [Nv][D], w [Nv].
 * Any output may be NULL. */
avs_status avs_get_tree(avs_ctx *ctx, int *level, int *base, uint32_t *key, double *xi, double *w);

/* f copy-out / copy-in in FP64 [Nc][nA][Nv] (parity and checkpoints). */
avs_status avs_get_f(avs_ctx *ctx, double *f, int is_device);
avs_status avs_set_f(avs_ctx *ctx, const double *f, int is_device);

/* FP64 copy-out of f for a list of cells only (sampled parity at full size,
 * where a whole FP64 copy would not fit in host memory).  cells: host array
 * of ncells indices, each in [0, Nc) (else AVS_EINVAL before any work); out:
 * host [ncells][nA][Nv].  Allocates and frees a device buffer of
 * ncells * nA * Nv doubles (AVS_ENOMEM if it cannot); blocking. */
avs_status avs_get_f_cells(avs_ctx *ctx, const int *cells, int ncells, double *out);

/* Criterion values M_k, as avs_criterion, for caller-owned device arrays and
 * without allocating any device memory.  The paper has no counterpart: this is
 * a library service for callers that cannot allocate on demand, such as an
 * embedder whose device memory belongs to another allocator (a caching pool, a
 * fixed budget) or a latency-sensitive loop that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree.  It needs no context.
 *   f [Nc][nA][Nv] (packed, nA = 2 in 2D, 1 in 3D), xi [Nv][dim], w [Nv],
 *   Wc [Nc][dim+2] conserved, M_out [Nv]: all device pointers on the current
 *   device; work is enqueued on cuda_stream (NULL: default stream).
 * Scratch lives in fixed device arrays of the library: at most 262144 cells
 * and 131072 nodes (about 11 MiB, held by every GPU that loads the library
 * until exit); larger inputs return AVS_ECAPACITY with a message on stderr.
 * All calls share that scratch and it keeps the last call's contents (each call
 * resets what it needs); calls that overlap on the GPU race and must be
 * ordered.  The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress) and should come before any stream capture; after a
 * device reset the next call looks it up again.  The status covers this
 * call's own launches (an error pending from earlier code is cleared first).
 * Errors: EINVAL (bad argument), ECAPACITY, ECUDA. */
avs_status avs_criterion_noalloc(int dim, int Nc, int Nv, const double *f, const double *xi, const double *w,
                                 const double *Wc, double *M_out, void *cuda_stream);

/* ---- learned proposer (not in the paper) ------------------------------------
 * An MLP 8 -> 64 -> 64 -> 4 (ReLU, ReLU, logits), BF16 tensor-core forward and
 * backward passes with FP32 accumulation and FP32 master weights.  From eight
 * per-cell features (log rho, the velocity components over sqrt(R T_ref) (in
 * 2D the third slot holds |q|/(rho (RT)^1.5)), log T, log of the mean free
 * path of Eq. 4 over the cell size, the largest relative jumps of rho and T to
 * the face neighbours; for the Rykov model T is the translational temperature
 * T_t and q the total heat flux q_t + q_r) it predicts four per-cell labels of
 * the Sec. 3.4 criterion (split witness, dominant, near-dominant, merge
 * blocker).  With cfg.learned = 1, avs_adapt evaluates the criterion only on
 * the cells whose dominant logit exceeds the threshold (the check set: the cell
 * attaining M_k decides both the split and the merge test of node k);
 * every learned_full_every-th adaptation it also runs the full criterion,
 * counts the nodes whose decision the check set got wrong, takes labels from
 * it and trains.  The check set keeps a budgeted fraction of the cells by
 * dominant logit (initially 25 %); the budget doubles after a full step that
 * found more than 1 % of the nodes missed and shrinks by 20 % after one that
 * found none.  Parameters: AVS_MLP_NPARAM floats laid out
 * W1[64][8], b1[64], W2[64][64], b2[64], W3[4][64], b3[4] (weights [out][in]). */
#define AVS_MLP_NPARAM 4996
avs_status avs_mlp_set_params(avs_ctx *ctx, const float *params);     /* host */
avs_status avs_mlp_get_params(avs_ctx *ctx, float *params);           /* host */
/* logits [n][4] of features X [n][8]; host buffers. */
avs_status avs_mlp_forward(avs_ctx *ctx, const float *X, int n, float *logits);
/* Mean binary cross-entropy over n x 4 outputs and its gradient (host
 * buffers, grad_out [AVS_MLP_NPARAM] nullable); lr > 0 also applies one SGD
 * step to the master weights. */
avs_status avs_mlp_grad(avs_ctx *ctx, const float *X, const float *Y, int n, float lr, float *grad_out,
                        float *loss_out);
/* Features [Nc][8] and criterion labels [Nc][4] of the current state (host, nullable). */
avs_status avs_features(avs_ctx *ctx, float *X_out, float *Y_out);
/* iters SGD steps on the current state's features and labels; last loss out. */
avs_status avs_mlp_train(avs_ctx *ctx, int iters, float lr, float *loss_out);
/* The check set of the last avs_adapt call of the learned form: *n_out = its
 * number of cells, or -1 when that call evaluated no check set (plain form,
 * untrained network); cells_out (host, nullable, room for Nc ints) receives
 * the cell indices in no particular order.  For tests and diagnostics: the
 * criterion restricted to these cells gives the decisions of a learned
 * adaptation and, on a full one, the misses it reports. */
avs_status avs_mlp_check_set(avs_ctx *ctx, int *cells_out, int *n_out);

/* The adaptive parameters of Sec. 3.5 for a flow.  With sigma = sqrt(R T):
 * T_0 = T_inf (1 + (gamma - 1)/2 Ma^2) (Eq. totaltemperature); R_dv =
 * rdv_sigma sigma_0; the domain is the square (cube) of half-width R_dv
 * centred at 0.4 U_inf; L_max = the least L with 2^L >= 2 R_dv / h_std;
 * L_w = L_max if T_w / T_inf < 4, else L_max - 1; L_min = 4 for D = 2 and
 * Ma > 5, else 3 (at most L_max); L_sep = max(L_min, L_w - 1).  The base
 * forest is the mesh of level L_min (2^L_min elements per axis, so the
 * paper's root element split L_min times); the tree then reaches L_max.
 * Zones, levels counted from L_min: free stream (centre U_inf, radius
 * 3 sigma_inf, L_max), stationary (centre 0, radius 3 sigma_w, L_w) and, with
 * `separated`, the ring 3 sigma_w .. 5 sigma_w about 0 (L_sep); elsewhere
 * L_min.  init_refine = max(0, L_w - 1 - L_min) (step 2 splits the root
 * L_w - 1 times).  C1 = 13.749 Ma^-1.465 (Eq. C1_Ma), C2 = 3.3546e-4 C1
 * (Eq. c2c1).  Writes dim, base, vlo, vhi, max_refine, nzones, zones,
 * zone_outside_level, init_refine, C1 and C2 of *cfg and nothing else.  Host
 * only, no context.  Errors: EINVAL (dim, Ma <= 0, gamma <= 1, R, T_inf,
 * T_w, h_std or rdv_sigma <= 0, zero direction). */
avs_status avs_paper_parameters(const avs_flow_spec *spec, avs_config *cfg);

/* Self-test of the bounded grid barrier that the implicit macroscopic sweep
 * uses between colour passes: one cooperative launch of `blocks` blocks
 * (1..number of SMs) passes `rounds` barriers; with short_by > 0 the last
 * barrier waits for short_by arrivals that never come, so each block gives up
 * after its poll limit (about a second) and the call returns AVS_ETIMEOUT with
 * the context still usable.  *passed (host) = barriers passed, summed over
 * blocks.  Blocking.  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
avs_status avs_grid_barrier_check(avs_ctx *ctx, int blocks, int rounds, int short_by, int *passed);

/* Self-test of the bounded mbarrier wait that the staged face and cell
 * kernels use for their asynchronous bulk copies: one block initialises an
 * mbarrier; with arrive = 1 one thread issues a 128-byte bulk copy into
 * shared memory that completes it, with arrive = 0 nothing ever does, so the
 * wait gives up after its limit (about a second), sets the error bit of the
 * staged copies and the call returns AVS_ETIMEOUT with the context still
 * usable.  *completed (host) = 1 when the copy arrived and its 128 bytes
 * equal the source's.  Blocking.  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
avs_status avs_stage_wait_check(avs_ctx *ctx, int arrive, int *completed);

/* Measured FMA throughput of the current GPU (GFLOP/s, 2 flops per FMA):
 * kind 0 FP32, 1 FP64, 2 FP32 pairs with the packed two-lane FMA.  Independent
 * multiply-add chains, timed with events; AVS_EINVAL for another kind.  A
 * measurement utility for the ALU rooflines; the paper has no counterpart. */
avs_status avs_measure_fma_peak(int kind, int iters, double *gflops);

/* Number of kernels this context has launched so far (all entry points). */
uint64_t   avs_kernel_launches(const avs_ctx *ctx);

/* Waits for the context's stream and reports a pending device error. */
avs_status avs_sync(avs_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
