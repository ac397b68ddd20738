/*
 * bid.h -- C ABI of the GB300 bidomain time-step library.
 *
 * The library solves, at every time step, the linear system of the coupled
 * heart-and-torso bidomain model of C. Pierre, "Preconditioning the bidomain
 * model with almost linear complexity" (arXiv 1711.08708):
 *
 *   Lambda X = Y,  Lambda = [[S_1, Pi^T S_i], [S_i Pi, gamma M_H + S_i]],
 *   int_Omega U = 0                                      (Sec. 3.2, eq. system)
 *
 * by FP64 preconditioned conjugate gradients with the block-LU preconditioner
 * P_Lambda = L_P U_P (Def. 5.1, eq. prec-def / prec2), P_1 built from S_1 and
 * P_K from the monodomain matrix K_m = gamma M_H + S_m (Sec. 5.2), both as
 * hierarchical (nested-dissection, low-rank compressed) Cholesky factors with
 * accuracy eps (Sec. 5.3).  The reaction term is the Mitchell-Schaeffer model.
 *
 * Conventions for every entry point:
 *  - Vectors passed to the solver calls are DEVICE pointers (cudaMalloc'd or
 *    torch tensors' data), FP64, in the library's node numbering: heart nodes
 *    first (hypothesis H1, Sec. 3.1), so U = X[0:N], V = X[N:N+N_H] and
 *    Pi U = U[0:N_H].  bid_get_perm gives library index -> mesh node.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued on it; calls documented as blocking synchronise it before return.
 *  - Every function returns BID_OK or an error code and never aborts; a
 *    message for the last error of the calling thread is at bid_last_error().
 *  - Handles own their device memory and free it in bid_destroy_*.  Nothing is
 *    allocated per solve or per step: work vectors live in the preconditioner.
 *  - Handles are not thread safe: one thread (and one stream at a time) per
 *    preconditioner handle.
 *  - The PCG loop of bid_solve / bid_step (and of the batched calls) runs as a
 *    CUDA graph whose WHILE condition is set on the device, so one solve costs
 *    one graph launch and one host read.  With the environment variable
 *    BID_PCG_GRAPH=0 (read once per process) the host launches the same
 *    kernels in the same order instead and reads the condition after every
 *    iteration: same results, for profilers that do not see kernels inside
 *    graphs with conditional nodes.
 *  - Other switches, read once per process (defaults are the measured best):
 *    BID_MASK=0      the preconditioner's second P_1 solve computes every
 *                    cluster instead of taking the clusters without heart
 *                    nodes from the all-ones forward results (equal up to
 *                    rounding);
 *    BID_PDL=0       the factor-solve kernels launch in plain stream order
 *                    instead of with programmatic dependent launch;
 *    BID_TREE=1      a range of flat levels runs in two dataflow launches per
 *                    solve (BID_TREE_FROM first level, default 1;
 *                    BID_TREE_SMEM shared-memory cap, default 32768);
 *    BID_UPPER=1     the top levels run in persistent cooperative launches;
 *    BID_FLATP=1     persistent double-buffered launches on the flat levels
 *                    with more groups than resident CTAs instead of one CTA
 *                    per group;
 *    BID_MERGE_MIN=n in the cluster tree, every subtree of at least n nodes has
 *                    its separator merged with its two children's (half as many
 *                    upper levels; read at preconditioner build);
 *    BID_UP_BROWS=n  target rows per warp of the large-cluster backward tasks
 *                    (default 512; read at preconditioner build);
 *    BID_MID_BYTES=n largest block (bytes) of a large cluster solved by one CTA
 *                    with its whole block in shared memory (default 98304; 0:
 *                    every large cluster takes the chunked kernels; read at
 *                    preconditioner build);
 *    BID_WIDE_BYTES=n factor bytes per CTA of a large cluster split in column
 *                    slices over a thread-block cluster (default 163840; 0:
 *                    none; read at preconditioner build);
 *    BID_ROOT_GRAM=0 the root cluster keeps its forward and backward passes
 *                    instead of one product with its Gram matrix (read at
 *                    preconditioner build);
 *    BID_GPU_FRONT_NF=n  smallest front factorised on the GPU (default 1024);
 *    BID_GROUP_BYTES / BID_GROUP_BYTES_LEAF  flat group size in bytes
 *                    (1024..65536, default 12288), read at preconditioner build.
 *    Results are the same with every setting: bit for bit, except that the
 *    masked solve's clusters computed in full (all of them with BID_MASK=0,
 *    those of the levels that BID_TREE or BID_UPPER take over) round
 *    differently, and that BID_MID_BYTES, BID_WIDE_BYTES and BID_ROOT_GRAM
 *    change the summation order of the large clusters they move between kinds
 *    of kernels.
 */
#ifndef BID_H
#define BID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BID_OK 0
#define BID_EINVAL 1     /* bad argument: size, NULL pointer, non-positive parameter */
#define BID_ENOCONV 2    /* max_iter reached; X holds the last iterate */
#define BID_ESTAGNATE 3  /* residual not finite (NaN/Inf in the data) */
#define BID_ECUDA 4      /* a CUDA runtime call failed */
#define BID_ETIMEOUT 5   /* a bounded device wait expired */
#define BID_ENOMEM 6     /* host or device allocation failed */

/* storage precision of the hierarchical factors (Sec. 5.3 precision form) */
#define BID_FP64 0
#define BID_FP32 1
#define BID_BF16 2

/* elliptic solvers of P_1 and P_K (the block-LU preconditioner admits any
 * good preconditioners of S_1 and K, Sec. 5.2) */
#define BID_ELLIPTIC_HCHOL 0 /* hierarchical (nested-dissection, eps-compressed)
                                Cholesky factors (Sec. 5.3) */
#define BID_ELLIPTIC_MG 1    /* one geometric-multigrid V-cycle: the mesh nodes must
                                be the points of a regular lattice and its
                                simplices the Kuhn simplices of the cells (2D:
                                squares cut along the (+1, +1) diagonal; 3D: six
                                tetrahedra around the (+1, +1, +1) diagonal); coarse
                                level = points with all indices even, P1
                                interpolation, Galerkin coarse operators,
                                Chebyshev smoothing of degree 2 before and after
                                the correction, dense inverse on the coarsest
                                level; FP64; eps, leaf and block are not used */

/* time schemes of bid_step (Sec. 3.2 and the remark on the time
 * discretisation: a scheme changes Step 1 and the coefficient of M_H in
 * Lambda, which keeps its structure) */
#define BID_SCHEME_EULER 0   /* semi-implicit Euler of the resolution algorithm
                                (Sec. 3.2): Lambda with gamma = chi Cm / dt */
#define BID_SCHEME_CN 1      /* Crank-Nicolson diffusion, reaction explicit at t^n:
                                Lambda(2 gamma) X^{n+1} = [0; M_H (2 gamma V^n -
                                2 chi (I_ion - I_st)) - S_i (Pi U^n + V^n)] */
#define BID_SCHEME_STRANG 2  /* Strang splitting: Heun reaction half step, Crank-
                                Nicolson diffusion step (its midpoint Z solves
                                Lambda(2 gamma) Z = [0; 2 gamma M_H V*], V = 2 Z_V -
                                V*), Heun reaction half step; U returned is Z_U, the
                                extracellular potential at the middle of the step */

/* Mesh of Omega with the heart sub-mesh (Sec. 3.1, hypothesis H1).  All arrays
 * are HOST memory, borrowed for the duration of bid_assemble only. */
typedef struct bid_mesh {
    int32_t dim;              /* 2 or 3 */
    int64_t n_nodes;
    int64_t n_elems;
    const double* coords;     /* [n_nodes * dim], cm */
    const int32_t* elems;     /* [n_elems * (dim+1)] P1 simplices, mesh node ids */
    const int32_t* region;    /* [n_elems]: 1 heart (T_H), 0 torso (T) */
    const double* fibre;      /* [n_elems * dim * dim] row-major frame whose
                                 columns are the local axes (fibre, sheet, normal) */
} bid_mesh;

/* Model parameters (Sec. 2; Mitchell-Schaeffer reaction term). */
typedef struct bid_params {
    double sigma_i[3];        /* g_i^l, g_i^t, g_i^n  (mS/cm; n unused in 2D) */
    double sigma_e[3];        /* g_e^l, g_e^t, g_e^n */
    double sigma_T;           /* isotropic torso conductivity k (mS/cm) */
    double chi;               /* membrane surface-to-volume ratio A_m (cm^-1) */
    double Cm;                /* membrane capacitance (uF/cm^2) */
    double tau_in, tau_out, tau_open, tau_close, v_gate;   /* ms, v_gate normalised */
    double v_rest, v_peak;    /* mV: w = (v - v_rest)/(v_peak - v_rest) */
    double stim_t_on, stim_t_off;  /* stimulus window [on, off) in ms */
    int32_t mass_lumped;      /* must be 1: row-sum (diagonal) mass matrices */
} bid_params;

typedef struct bid_system bid_system;    /* assembled S_1, S_i, M, M_H on the device */
typedef struct bid_precond bid_precond;  /* P_1, P_K factors + PCG work vectors */

/* Options of the preconditioner build (defaults via bid_precond_opts_default). */
typedef struct bid_precond_opts {
    double dt;                /* time step (ms); gamma = chi * Cm / dt (Sec. 3.2) */
    double eps;               /* low-rank truncation accuracy (Sec. 5.3); 0 = exact */
    int32_t precision;        /* BID_FP64 | BID_FP32 | BID_BF16 factor storage */
    int32_t leaf_size;        /* nested-dissection leaf: max nodes per leaf cluster (4..4096) */
    int32_t block;            /* rows of a low-rank boundary group (8..256) */
    int32_t n_threads;        /* host threads for the build (0 = all) */
    int32_t scheme;           /* BID_SCHEME_*: time scheme of bid_step; the factors and
                                 bid_solve use gamma = chi Cm / dt (EULER) or twice
                                 that (CN, STRANG) */
    int32_t elliptic;         /* BID_ELLIPTIC_*: how P_1 and P_K are applied */
    int32_t gpu_build;        /* 1 (default): the dense work of the large fronts (at
                                 least 1024 rows; BID_GPU_FRONT_NF overrides) of the
                                 hierarchical factors runs on the GPU (FP64 Cholesky,
                                 inverse and products, the same factors up to rounding);
                                 the symbolic tree, the small fronts and the low-rank
                                 compression stay on the host; 0: host only */
} bid_precond_opts;

typedef struct bid_precond_stats {
    int64_t n1, nk;                    /* sizes of the S_1 and K_m factors */
    int64_t supernodes1, supernodesk;
    int32_t levels1, levelsk;          /* tree heights (launches per triangular pass) */
    int64_t dense_entries, lowrank_entries;  /* stored factor entries, both factors */
    int64_t factor_bytes;              /* algorithmic factor bytes of one P_Lambda^-1:
                                          two P_1 solves and one P_K solve */
    int64_t bytes_p1, bytes_pk;        /* stored bytes read by one forward+backward
                                          pair (including alignment padding) */
    int64_t alg_bytes_p1, alg_bytes_pk;  /* the same without padding (nonzero
                                          dense entries and low-rank factors) */
    int64_t lowrank_blocks, dense_blocks;
    double build_seconds;
    int32_t dataflow_levels1, dataflow_levelsk;  /* levels solved by the two dataflow
                                          launches per pass (0: one launch per level, the
                                          default; BID_TREE=1 in the environment turns
                                          them on) */
    int32_t dataflow_first1, dataflow_firstk;    /* the first of those levels */
    int32_t large_levels1, large_levelsk;  /* tree levels holding large clusters (solved
                                          by the chunked large-cluster kernels) */
    int64_t masked_dead1, masked_clusters1;  /* clusters of P_1 whose forward results the
                                          masked second P_1 solve takes from the all-ones
                                          solve, and all clusters (0, 0 with BID_MASK=0) */
    int64_t alg_bytes_p1_masked;       /* algorithmic bytes of one masked P_1 solve: the
                                          forward blocks of the live clusters and the whole
                                          backward pass (alg_bytes_p1 with BID_MASK=0) */
    int32_t flatp_levels1, flatp_levelsk;  /* flat levels solved by persistent double-
                                          buffered launches (more groups than resident
                                          CTAs), forward pass; 0 unless BID_FLATP=1 */
    int64_t mid_clusters1, mid_clustersk;  /* large clusters solved by one CTA each with
                                          their whole block in shared memory (at most
                                          BID_MID_BYTES bytes, default 96 KiB; 0 turns
                                          them off); the other large clusters take the
                                          chunked kernels */
    int64_t wide_clusters1, wide_clustersk;  /* large clusters solved by a thread-block
                                          cluster of CTAs, each holding a column slice of
                                          the block in shared memory (at most
                                          BID_WIDE_BYTES bytes per CTA, default 160 KiB; 0
                                          turns them off); counted where the device runs
                                          them (the host replay: where they are built) */
    int64_t gram_pivots1, gram_pivotsk;  /* pivots of the root cluster whose forward and
                                          backward passes are one product with its Gram
                                          matrix M^T M (0: none; BID_ROOT_GRAM=0 turns it
                                          off) */
} bid_precond_stats;

typedef struct bid_solve_info {
    int32_t iters;            /* P_Lambda^-1 applications after the initial one */
    int32_t status;           /* BID_OK / BID_ENOCONV / BID_ESTAGNATE */
    int32_t restarts;         /* true-residual restarts (at most 1) */
    double relres;            /* recurrence residual ||r||/||Y|| at exit */
    double relres_true;       /* ||Y - Lambda X||/||Y|| recomputed at exit */
} bid_solve_info;

/* Assemble S_1 (sigma_1 = sigma_i + sigma_e on H, sigma_T on T), S_i, lumped
 * M and M_H with P1 elements (Sec. 3.1) and S_m (sigma_m, Sec. 5.2); reorder the
 * nodes heart-first; upload to the current CUDA device.  Blocking.
 * Errors: BID_EINVAL (dim, sizes, node ids out of range, no heart element,
 * non-positive conductivity, mass_lumped != 1), BID_ENOMEM, BID_ECUDA. */
int bid_assemble(const bid_mesh* mesh, const bid_params* params, bid_system** out);

/* Sizes: N, N_H and stored non-zeros of S_1 and S_i (any pointer may be NULL). */
int bid_system_sizes(const bid_system* s, int64_t* N, int64_t* NH,
                     int64_t* nnz_s1, int64_t* nnz_si);

/* perm[k] = mesh node of library index k (host array of N entries). */
int bid_get_perm(const bid_system* s, int64_t* perm);

/* Lumped mass diagonals (host arrays, N and N_H entries; either may be NULL). */
int bid_get_mass(const bid_system* s, double* m, double* mH);

void bid_precond_opts_default(bid_precond_opts* o);

/* Build P_Lambda for time step dt (Def. 5.1 with Sec. 5.2-5.3): the nested-
 * dissection Cholesky factors of S_1 (the last U unknown pinned, which makes
 * the factor an exact pseudo-inverse solver on 1^perp) and of K_m, in explicit
 * inverse-block form with eps-truncated low-rank blocks, stored in `precision`.
 * Host build (OpenMP), then upload.  Blocking.
 * Errors: BID_EINVAL (dt <= 0, eps < 0, bad precision/leaf/block), BID_ENOMEM,
 * BID_ECUDA. */
int bid_precond_build(bid_system* s, double dt, double eps, int precision,
                      bid_precond** out);
/* The same with every option (leaf size, low-rank block rows, host threads,
 * time scheme, elliptic solver); defaults from bid_precond_opts_default.
 * With BID_ELLIPTIC_MG the build makes the multigrid hierarchies instead of
 * the factors (EINVAL when the mesh is not a Kuhn lattice or precision is not
 * BID_FP64); the stats then give the hierarchies' levels (levels1, levelsk),
 * their stored matrix entries (dense_entries) and the algorithmic bytes of
 * one V-cycle (alg_bytes_p1, alg_bytes_pk).  The build also takes the all-ones
 * forward results of P_1 used by the masked second P_1 solve (one extra solve,
 * skipped with BID_MASK=0). */
int bid_precond_build_ex(bid_system* s, const bid_precond_opts* opts,
                         bid_precond** out);
/* Factor statistics of P (host struct, filled at build; no device work).
 * Errors: BID_EINVAL (NULL argument). */
int bid_precond_get_stats(const bid_precond* P, bid_precond_stats* st);

/* y = Lambda(gamma) x (eq. system); x, y device, N + N_H each, distinct. */
int bid_apply_lambda(const bid_system* s, double gamma, const double* x, double* y,
                     void* stream);

/* z = P_Lambda^-1 r (eq. prec2): Z1 = P_1^-1 p r_U, T = r_V - S_i Pi Z1,
 * Z2 = P_K^-1 T, Z1 -= P_1^-1 Pi^T S_i Z2, where p projects onto 1^perp.  r and
 * z device, N + N_H each, distinct.  The U block of z is defined up to an
 * additive constant (Lambda annihilates constants, Prop. 1). */
int bid_apply_precond(bid_precond* P, const double* r, double* z, void* stream);

/* Solve x = P_1^-1 (b - mean(b)) (which = 1: S_1 factor, N entries) or
 * x = P_K^-1 b (which = 2: K_m factor, N_H entries).  Device vectors. */
int bid_apply_factor(bid_precond* P, int which, const double* b, double* x, void* stream);

/* Same result as bid_apply_factor, but the call allocates nothing.  (The paper
 * has no counterpart: this is a library service.)  It is meant for callers
 * that cannot call cudaMalloc at the moment they solve: a real-time loop that
 * must not pay for the allocator's implicit device synchronisation, or a host
 * application that hands the library a fixed memory budget up front and
 * forbids device allocations afterwards.
 * bid_apply_factor itself only uses buffers made by bid_precond_build, but
 * this variant takes its scratch (the forward-pass, update, rank, partial-sum
 * and ticket buffers) from one static device array of 2^21 doubles (16 MiB)
 * that every GPU loading this library holds until the process exits.
 * Limit: a factor whose scratch (its size plus its update, rank and
 * partial-sum entries) exceeds that array is rejected with BID_EINVAL and a
 * message; use bid_apply_factor for it.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The array is shared by all
 * calls and keeps the last call's contents (the tickets it needs at zero are
 * cleared on each call), so calls that overlap on the GPU -- on different
 * streams, or from different threads -- race: serialise them.  Device
 * pointers, stream semantics and which / b / x as for bid_apply_factor; as
 * there, an expired bounded device wait is recorded in P's error word (built
 * with P, so nothing is allocated) and reported as BID_ETIMEOUT by the next
 * bid_solve / bid_step on P.  The cached address belongs to the device's
 * current context: after a device reset (which also invalidates every handle
 * of this library) do not call this entry point again in the process. */
int bid_apply_factor_noalloc(bid_precond* P, int which, const double* b, double* x,
                             void* stream);

/* Kernel classes of one PCG time step, each timed alone with CUDA events on
 * `stream` (one warm-up launch, then `reps` launches back to back; ms[c] is
 * the mean milliseconds of one launch of class c).  The classes, in the order
 * of ms (BID_PROFILE_CLASSES entries):
 *   0 Lambda product (eq. system), fused <p, q> and sum(q_U);
 *   1 P_1 solve (forward and backward passes of the S_1 factor);
 *   2 masked P_1 solve (the preconditioner's second P_1 application, eq. prec2);
 *   3 P_K solve (the K_m factor);
 *   4 the S_i products and the update of the block-LU chain (eq. prec2);
 *   5 PCG vector kernels of one iteration (<r, z>, p update, x and r updates
 *     with the projection, convergence test);
 *   6 residual Y - Lambda X with the projection (start and end of a solve);
 *   7 Step 1 + Step 3 (right-hand side and gate update);
 *   8 normalisation (proof of Prop. 1).
 * The call overwrites P's work vectors and scalars (inputs are a fixed finite
 * pattern), so it must not run while a solve on P is in flight; the next
 * bid_solve / bid_step starts afresh.  Blocking.  Errors: BID_EINVAL (NULL P
 * or ms, reps < 1), BID_ECUDA. */
#define BID_PROFILE_CLASSES 9
int bid_profile_classes(bid_precond* P, int reps, double* ms, void* stream);

/* Step 2 (eq. system): PCG on Lambda from the guess in X, stopping when the
 * recurrence residual ||r||_2/||Y||_2 < tol (Sec. 6.2); the true residual is
 * then recomputed and PCG restarted once if it is above tol; X is finally
 * normalised so that (M U, 1) = 0 (proof of Prop. 1).  Y must lie in
 * Ran(Lambda) (U block summing to zero); the U block of every residual is
 * projected onto 1^perp.  Y and X device (N + N_H), distinct.  Blocking: info
 * (may be NULL) is filled before return.  Returns BID_ENOCONV after max_iter. */
int bid_solve(bid_system* s, bid_precond* P, const double* Y, double* X,
              double tol, int max_iter, bid_solve_info* info, void* stream);

/* The resolution algorithm (Sec. 3.2) for n_steps steps from time t0:
 * Step 1 and Step 3 fused (Y from (V^n, W^n); W^{n+1} = W^n + dt g(V^n, W^n)),
 * Step 2 by bid_solve with guess (U^n, V^n).  U (N), V (N_H), h (N_H) device,
 * updated in place.  Ist: device per-heart-node stimulus amplitude (uA/cm^2)
 * applied while t in [stim_t_on, stim_t_off), or NULL.  iters_out: host array
 * of n_steps PCG iteration counts, or NULL.  Blocking.
 * The preconditioner's scheme (bid_precond_opts.scheme) selects the time
 * scheme: BID_SCHEME_CN replaces Step 1 by its Crank-Nicolson right-hand side
 * (one fused kernel, which reads U^n: U must satisfy the elliptic equation
 * with V, as it does after any step and for the resting state U = 0,
 * V = v_rest); BID_SCHEME_STRANG runs the reaction half steps (stimulus
 * sampled at t, t + dt/2 and t + dt) around the Crank-Nicolson diffusion
 * solve and returns in U the extracellular potential at t + dt/2 (U on input
 * is only the solve's initial guess). */
int bid_step(bid_system* s, bid_precond* P, double* U, double* V, double* h,
             const double* Ist, double t0, int n_steps, double tol, int max_iter,
             int* iters_out, void* stream);

/* Step 1 + Step 3 only: Y[0:N] = 0, Y[N:] = M_H (gamma V - chi (I_ion - I_st)),
 * h += dt g(V, h), with the stimulus on iff stim_on != 0.  Device pointers. */
int bid_rhs_gate(bid_precond* P, const double* V, double* h, const double* Ist,
                 int stim_on, double* Y, void* stream);

/* U <- U - (M U, 1)/(M 1, 1) on the U block of X (device, N + N_H or N). */
int bid_normalise(bid_precond* P, double* X, void* stream);

void bid_destroy_system(bid_system* s);
void bid_destroy_precond(bid_precond* P);
const char* bid_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads; used to report launches inside a timed region). */
int64_t bid_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Batched form: many independent problems ("slices", each assembled by
 * bid_assemble on its own mesh) advanced together, with the semantics of one
 * bid_solve / bid_step per slice.  Each phase of the method (Lambda product,
 * P_1 and P_K solves, vector updates, convergence test) is one kernel launch
 * over all slices, and the PCG loop of all slices is one CUDA graph whose
 * device-side WHILE condition runs until every slice has converged; a slice
 * that has converged is frozen (its iterate no longer changes).
 *
 * Combined layout: slice s owns entries [off[s], off[s+1]) of every combined
 * vector, laid out as that slice's own X ([U_s | V_s], N_s + N_H,s entries,
 * heart nodes first), so X_s = X + off[s]; its heart-indexed arrays (gates h,
 * stimulus Ist) are entries [hoff[s], hoff[s+1]) of the combined heart
 * arrays.  bid_batch_layout returns off and hoff.
 * ------------------------------------------------------------------------- */
typedef struct bid_batch bid_batch;

/* Build the batch: the factors of every slice (one nested-dissection tree per
 * slice; leaf[s] its leaf size, or opts->leaf_size for all when leaf is NULL;
 * dt, eps, precision, block, n_threads from opts) and the combined device
 * layout.  The systems are borrowed and must outlive the batch.  All slices
 * share the reaction and stimulus parameters (chi, Cm, Mitchell-Schaeffer
 * constants, stimulus window) and the dimension; conductivities and meshes
 * may differ.  Blocking.
 * Errors: BID_EINVAL (nslices < 1 or > 32767, NULL system, differing reaction
 * parameters or dimension, bad opts or leaf, more than 2^31 unknowns in
 * all), BID_ENOMEM, BID_ECUDA. */
int bid_batch_create(bid_system* const* systems, int nslices, const bid_precond_opts* opts,
                     const int32_t* leaf, bid_batch** out);
/* off, hoff: host arrays of nslices + 1 entries (either may be NULL). */
int bid_batch_layout(const bid_batch* B, int64_t* off, int64_t* hoff);
/* Factor statistics of the batch (both forests, all slices together). */
int bid_batch_get_stats(const bid_batch* B, bid_precond_stats* st);
/* bid_apply_factor for every slice at once on combined device vectors:
 * which = 1: x_U,s = P_1,s^-1 (b_U,s - mean(b_U,s)), which = 2:
 * x_V,s = P_K,s^-1 b_V,s; the other entries of x are not written. */
int bid_batch_apply_factor(bid_batch* B, int which, const double* b, double* x, void* stream);
/* bid_apply_precond for every slice (combined device vectors r, z). */
int bid_batch_apply_precond(bid_batch* B, const double* r, double* z, void* stream);
/* bid_solve for every slice: Y, X combined device vectors (distinct); info:
 * host array of nslices entries or NULL.  Returns the first error of any
 * slice (BID_ESTAGNATE before BID_ENOCONV); info tells which.  Blocking. */
int bid_batch_solve(bid_batch* B, const double* Y, double* X, double tol, int max_iter,
                    bid_solve_info* info, void* stream);
/* bid_step for every slice: X (combined state, U_s and V_s of each slice), h
 * (combined gates) and Ist (combined stimulus amplitudes or NULL) device,
 * updated in place; iters_out: host array of n_steps * nslices counts (step
 * major) or NULL.  Blocking. */
int bid_batch_step(bid_batch* B, double* X, double* h, const double* Ist, double t0,
                   int n_steps, double tol, int max_iter, int* iters_out, void* stream);
void bid_batch_destroy(bid_batch* B);

/* Leaf-size tuner: builds the preconditioner of s with each leaf size in
 * cands (other options from opts), times `reps` applications of
 * P_Lambda^-1 with CUDA events, and returns the fastest in *best and the mean
 * milliseconds per application of every candidate in ms_out (ncands entries,
 * may be NULL).  Results are cached in the process, keyed by the system's
 * sizes and the options: a repeated query returns at once.  Blocking. */
int bid_tune_leaf(bid_system* s, const bid_precond_opts* opts, const int32_t* cands,
                  int ncands, int reps, int32_t* best, double* ms_out);
/* Leaf sizes for a batch: the slices are grouped in classes of half an octave
 * of N; bid_tune_leaf runs on the slice of median N of each class and its
 * answer is given to the whole class.  leaf_out: host array of nslices
 * entries, ready for bid_batch_create.  Blocking. */
int bid_tune_batch_leaf(bid_system* const* systems, int nslices, const bid_precond_opts* opts,
                        const int32_t* cands, int ncands, int reps, int32_t* leaf_out);

/* ---------------------------------------------------------------------------
 * Learned initial guess.  A small convolutional network on the node grid of
 * a structured slice -- three 3 x 3 convolutions, 6 -> 32 -> 32 -> 2
 * channels, ReLU after the first two, zero padding -- maps the last three
 * steps' U and V (V - v_rest, zero outside the heart) -- as U^n, its last two
 * increments, V^n and its last two increments, each over a fixed scale -- to
 * the scaled increments of U and V at the next step.  PCG then starts from
 * (U^n + dU, V^n + dV) when that guess has a smaller initial residual than
 * the previous step (U^n, V^n), which stays the fallback.  The guess changes only the iteration count: the
 * solve and its stopping rule are those of bid_solve.  (The paper has no
 * counterpart; the network is trained on solves of the method itself.)
 * ------------------------------------------------------------------------- */
typedef struct bid_cnn bid_cnn;
typedef struct bid_guess bid_guess;

/* Number of network parameters, packed as W1 (32, 6, 3, 3), b1 (32),
 * W2 (32, 32, 3, 3), b2 (32), W3 (2, 32, 3, 3), b3 (2), row-major. */
int bid_cnn_nparams(void);
/* A network with He-style random weights from `seed` (FP32 master copy and
 * Adam moments on the device) and work buffers for batches of up to
 * max_pixels grid points.  Blocking. */
int bid_cnn_create(int max_pixels, uint64_t seed, bid_cnn** out);
/* Host FP64 arrays of bid_cnn_nparams() entries (stored as FP32; set resets Adam). */
int bid_cnn_set_params(bid_cnn* C, const double* params);
int bid_cnn_get_params(const bid_cnn* C, double* params);
/* Mean squared error of the network on a batch (over all points and both
 * outputs) and its gradient, computed by the library's own forward and
 * backward kernels in `precision` (BID_FP64: x, t are double; BID_FP32:
 * float).  x: device (B, H, W, 6) channels-last; t: device (B, H, W, 2).
 * loss (host) and grad (host, nparams, may be NULL).  Blocking. */
int bid_cnn_loss_grad(bid_cnn* C, int precision, const void* x, const void* t, int B, int H, int W,
                      double* loss, double* grad, void* stream);
/* One Adam step (lr, beta 0.9 / 0.999, eps 1e-8) on the FP32 gradient of
 * the batch (x, t float, device).  loss (host) may be NULL.  Blocking. */
int bid_cnn_train_step(bid_cnn* C, const float* x, const float* t, int B, int H, int W, double lr,
                       double* loss, void* stream);
/* Network output y (B, H, W, 2).  precision BID_FP64 (x, y double) or BID_FP32
 * (float): direct convolutions; BID_BF16: one grid (B = 1), x and y float,
 * BF16 weights and activations on the tensor cores with FP32 accumulation. */
int bid_cnn_forward(bid_cnn* C, int precision, const void* x, int B, int H, int W, void* y,
                    void* stream);
void bid_cnn_destroy(bid_cnn* C);

/* The guess for system s on an H x W grid: node_pixel (host, one entry per
 * mesh node) is a bijection of the nodes onto the grid points (row-major).
 * max_batch_pixels: training batch capacity (ncrops * crop^2).  The network
 * is borrowed.  Errors: BID_EINVAL (H W != N, not a bijection). */
int bid_guess_create(bid_system* s, bid_cnn* net, int H, int W, const int32_t* node_pixel,
                     int max_batch_pixels, bid_guess** out);
/* Append a solved state (U, V device, library numbering) to the history. */
int bid_guess_push(bid_guess* G, const double* U, const double* V, void* stream);
int bid_guess_reset(bid_guess* G);
/* `iters` Adam steps on random crops (ncrops of crop x crop points, origins
 * from `seed`) of the newest history entry: inputs the states n-1, n-2, n-3,
 * targets U^n - U^n-1 and V^n - V^n-1.  The first call fixes the scales (RMS
 * of U, V - v_rest and of both increments over the grid).  Needs four
 * states.  Blocking. */
int bid_guess_train(bid_guess* G, int ncrops, int crop, int iters, double lr, uint64_t seed,
                    double* loss, void* stream);
/* scales[4] (host): U, V - v_rest, dU, dV (0 before the first training call). */
int bid_guess_scales(const bid_guess* G, double* scales);
/* X0 = (U + dU, V + dV) from the last three history states (device, N + N_H). */
int bid_guess_predict(bid_guess* G, const double* U, const double* V, double* X0, void* stream);
/* use_dv: apply the predicted V increment (1, default) or keep V^n (0).
 * policy 0 (default): each step starts from the guess with the smaller
 * initial residual; policy 1: from the guess that needed fewer PCG
 * iterations on average so far (each guess is tried at least twice, and the
 * other one every 8th step).  Resets the iteration record. */
int bid_guess_configure(bid_guess* G, int use_dv, int policy);
/* bid_step with the learned guess (when three states are known; else the
 * previous step) chosen by the guess's policy; the new state is pushed to
 * the history.  stats (host, n_steps x 4 or NULL): PCG iterations, relative
 * initial residual of the previous-step guess and of the learned guess
 * (policy 0; 0 when not computed), and 1 when the learned guess was used.
 * Blocking. */
int bid_step_learned(bid_system* s, bid_precond* P, bid_guess* G, double* U, double* V, double* h,
                     const double* Ist, double t0, int n_steps, double tol, int max_iter,
                     double* stats, void* stream);
/* Frees the guess's device buffers (not the network it was created with). */
void bid_guess_destroy(bid_guess* G);

/* ---------------------------------------------------------------------------
 * Host-only entry points (no GPU needed).  They expose the host half of the
 * library -- the P1 assembly and the hierarchical factor build -- together
 * with a sequential host replay of the factor's level-by-level triangular
 * passes over exactly the packed blocks and tiles that the GPU kernels read.
 * They exist so that the host logic can be checked on machines without a GPU.
 * ------------------------------------------------------------------------- */
typedef struct bid_host_system bid_host_system;

/* Assemble on the host only (same arguments and errors as bid_assemble). */
int bid_host_assemble(const bid_mesh* mesh, const bid_params* params, bid_host_system** out);
/* Sizes of matrix `which` (0: S_1, 1: S_i, 2: S_m): rows and stored entries. */
int bid_host_csr_size(const bid_host_system* h, int which, int64_t* n, int64_t* nnz);
/* Copy matrix `which` in CSR form (ptr: n+1 entries, col/val: nnz entries),
 * library numbering; perm (N entries, may be NULL) and the lumped masses m
 * (N) and mH (N_H) (may be NULL) are copied too. */
int bid_host_csr(const bid_host_system* h, int which, int64_t* ptr, int32_t* col, double* val,
                 int64_t* perm, double* m, double* mH);
/* Build the factor of S_1 (which = 1, last U unknown pinned) or of
 * K_m = gamma M_H + S_m (which = 2) with the given eps / leaf / block, and
 * apply it on the host: x = P^-1 (b - mean(b)) for which = 1, x = P^-1 b for
 * which = 2.  The stored layout is the one built for `precision`; the replay
 * computes in FP64.  b and x are host arrays (N or N_H).  stats may be NULL. */
int bid_host_factor_solve(const bid_host_system* h, int which, double gamma, double eps,
                          int leaf, int block, int precision, const double* b, double* x,
                          bid_precond_stats* stats);
/* As bid_host_factor_solve, with the flat groups of a range of levels run in
 * the order of the dataflow solve kernels (the levels from `from` on whose
 * largest group needs at most smem_cap bytes of shared memory and that hold
 * no large cluster; smem_cap 0: level by level): forward, always the
 * highest-numbered group whose dependencies are complete, backward the
 * lowest-numbered, so that a missing dependency changes x.  With a complete
 * schedule x is bit-identical to bid_host_factor_solve's.  sched (5 entries,
 * may be NULL) receives the schedule's first and end level, groups, forward
 * and backward dependencies. */
int bid_host_factor_solve_dataflow(const bid_host_system* h, int which, double gamma, double eps,
                                   int leaf, int block, int precision, int smem_cap, int from,
                                   const double* b, double* x, bid_precond_stats* stats, int64_t* sched);
/* bid_host_factor_solve for which = 1 (P_1 of S_1) with b zero outside the
 * heart nodes (indices N_H .. N-1; EINVAL otherwise), replayed as the masked
 * solve: every cluster whose subtree holds no heart node sees the constant
 * input -mean(b) alone, so its forward results are -mean(b) times those of
 * the all-ones input, which the replay computes first and then copies
 * scaled.  Equal to bid_host_factor_solve's x up to rounding.  ndead (2
 * entries, may be NULL): dead clusters, all clusters. */
int bid_host_factor_solve_masked(const bid_host_system* h, double eps, int leaf, int block, int precision,
                                 const double* b, double* x, int64_t* ndead);
/* The batched factors on the host: the forest over nslices host systems
 * (combined layout as for bid_batch_create, leaf per slice or NULL for
 * `leaf_default`), replayed in FP64: which = 1 writes x_U,s = P_1,s^-1
 * (b_U,s - mean(b_U,s)), which = 2 writes x_V,s = P_K,s^-1 b_V,s (gamma as
 * given); other entries of x are left as they are.  b, x host arrays of the
 * combined length.  smem_cap, from and sched as for
 * bid_host_factor_solve_dataflow (smem_cap 0: level by level; sched may be
 * NULL).  masked != 0 (which = 1 only; b zero on every slice's torso nodes,
 * EINVAL otherwise): replayed as the masked forest solve, as in
 * bid_host_factor_solve_masked with each tree's own mean.  stats may be NULL. */
int bid_host_batch_factor_solve(const bid_host_system* const* hs, int nslices, int which,
                                double gamma, double eps, const int32_t* leaf, int leaf_default,
                                int block, int precision, int smem_cap, int from, int masked,
                                const double* b, double* x, bid_precond_stats* stats, int64_t* sched);
/* The multigrid V-cycle of BID_ELLIPTIC_MG on the host, in FP64 and in the
 * order of operations of the GPU kernels: which = 1: x = V_1(b - mean(b))
 * for S_1 (its hierarchy is singular: constants are its kernel), which = 2:
 * x = V_K(b) for K_m = gamma M_H + S_m.  b and x host arrays (N or N_H).
 * levels (may be NULL): the hierarchy's levels.  Errors: BID_EINVAL (bad
 * argument, mesh not a Kuhn lattice). */
int bid_host_mg_solve(const bid_host_system* h, int which, double gamma, const double* b, double* x,
                      int32_t* levels);
/* Frees a host system (NULL is ignored). */
void bid_host_destroy(bid_host_system* h);

#ifdef __cplusplus
}
#endif
#endif /* BID_H */
