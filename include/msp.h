/*
 * msp.h - C ABI of the GB300 library for the non-nested multilevel smoothed
 * Schwarz preconditioner of arXiv 2412.08981, applied inside right-
 * preconditioned FGMRES for P1 tetrahedral finite-element systems whose
 * coefficient k(x; mu) changes with a parameter vector mu while the mesh
 * hierarchy is reused.
 *
 * Conventions for every call:
 *   - Return value: an msp_status; MSP_OK (0) on success.  On failure the
 *     outputs are left untouched (msp_stats is always filled) and
 *     msp_last_error() returns a message for the calling thread.
 *   - Host pointers are caller-owned and only read during the call (they are
 *     copied).  "device" pointers are caller-owned CUDA device memory on the
 *     current device; the library never frees them.
 *   - Library-owned device memory (hierarchy, per-parameter instance) comes
 *     from msp_options.alloc / .free when given (the Python binding routes it
 *     to PyTorch's caching allocator), else from cudaMalloc / cudaFree.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is enqueued on it; calls that return results to the host
 *     (msp_solve, msp_solve_host) synchronise it.
 *   - Threads: different instances (of one hierarchy or several) may be used
 *     from different host threads at once, also when they share a stream
 *     (their work is then serialised on it).  One instance is used by one
 *     thread at a time.  A hierarchy is read-only after msp_load_hierarchy
 *     and may be shared by all threads; msp_free_hierarchy runs after its
 *     instances are freed.
 *   - Vectors on a level hold one FP64 entry per DoF (Dirichlet ones
 *     included): per mesh node in the node order of that level's
 *     msp_level_desc, three per node (DoF 3v + c) for linear elasticity.
 *   - Level 0 is the finest mesh M_0; level L-1 is the coarsest.
 */
#ifndef MSP_H_
#define MSP_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MSP_API __attribute__((visibility("default")))
#else
#define MSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum msp_status {
  MSP_OK = 0,
  MSP_PENDING = 1,             /* request still running (msp_poll) */
  MSP_ERR_INVALID = -1,        /* bad argument or mesh; nothing was changed */
  MSP_ERR_OOM = -2,            /* allocation failed or memory budget exceeded */
  MSP_ERR_NOT_CONVERGED = -3,  /* FGMRES hit max_it or broke down; x holds the last iterate */
  MSP_ERR_TIMEOUT = -4,        /* a bounded wait gave up */
  MSP_ERR_CUDA = -5,           /* a CUDA runtime call failed */
  MSP_ERR_INTERNAL = -6        /* a zero/non-finite pivot or a device-side check failed */
} msp_status;

/* Precision of the subdomain LU factors and their triangular solves.  The
 * outer FGMRES, every SpMV, the transfers and the directly solved coarsest
 * level stay FP64.
 *   MSP_F64 : factorisation and solves in FP64
 *   MSP_F32 : factorisation, storage and solves in FP32
 *   MSP_BF16: factorisation in FP32, factors rounded (to nearest even) to BF16
 *             for storage; the solves read BF16 and accumulate in FP32
 *   MSP_F64_TC: FP64 factors and solves as MSP_F64; on levels factored in one
 *             persistent launch, the panel and trailing products of every tile
 *             step run on the BF16 tensor cores, exactly, by splitting each
 *             operand row into eight 7-bit digits scaled to its largest entry
 *             (Ozaki's scheme; 36 digit-pair products, exact FP32 group sums,
 *             64-bit integer combination): every product entry is within
 *             2^-48 K max|a_r| max|b_c| of the exact one (worst case), below the
 *             worst case of an FP64 dot product of length K (K 2^-53 sum|a||b|).  Diagonal tiles and the tile steps
 *             of the other levels stay on the FP64 pipe. */
typedef enum msp_precision { MSP_F64 = 0, MSP_F32 = 1, MSP_BF16 = 2, MSP_F64_TC = 3 } msp_precision;

/* Coefficient family k(x; mu), evaluated at each tet centroid x_c:
 *   MSP_K_CONST : k = 1
 *   MSP_K_COSEXP: k = exp(s * sum_{j=1..8} mu_j * 0.5 * cos(pi * a_j . x_c)),
 *                 a_j integer wave vectors (msp_options.wave), s = coef_scale. */
typedef enum msp_coef { MSP_K_CONST = 0, MSP_K_COSEXP = 1 } msp_coef;

/* Right-hand side f of -div(k grad u) = f, integrated with the vertex rule
 * b_a = sum_{T containing a} f(x_a) |T| / 4 (0 on Dirichlet nodes):
 *   MSP_F_ONE  : f = 1
 *   MSP_F_SINES: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
 * For linear elasticity (MSP_PDE_ELASTICITY), per displacement field c:
 *   MSP_F_ONE  : f = (0, 0, -1), a unit body force along -z
 *   MSP_F_SINES: the force whose solution with k = 1 is u = (s, s, s),
 *                s = sin(pi x) sin(pi y) sin(pi z):
 *                f_c = 3 pi^2 mu_L s - (lambda_L + mu_L) sum_d d_c d_d s */
typedef enum msp_load { MSP_F_ONE = 0, MSP_F_SINES = 1 } msp_load;

/* The PDE and its DoF distribution (Section 2.1, the mesh perspective
 * M = (K, N)):
 *   MSP_PDE_POISSON   : -div(k grad u) = f, one DoF per vertex, N = (1,0,0,0);
 *   MSP_PDE_ELASTICITY: linear elasticity -div sigma(u) = f with
 *       sigma = k(x; mu) (2 mu_L eps(u) + lambda_L tr(eps(u)) I), the Lame
 *       parameters of a unit Young's modulus and Poisson ratio
 *       msp_options.poisson_ratio; three displacement fields per vertex,
 *       N = (3,0,0,0), DoF 3v + c for field c of vertex v.  A Dirichlet vertex
 *       fixes its three fields.  The transfers are split by field: P (x) I_3,
 *       the field-splitting interpolation I = sum_f R_f^T I_f R~_f of
 *       Section 2.1 with the scalar barycentric P for every field.
 *   MSP_PDE_POISSON_P2: -div(k grad u) = f with continuous piecewise-quadratic
 *       (P2) Lagrange elements: one DoF at every vertex and one at the midpoint
 *       of every edge, N = (1,1,0,0).  DoF order: vertex 0, then its edges
 *       (0, b) to higher-numbered vertices b in ascending b, then vertex 1 and
 *       its edges (1, b), b > 1, and so on (the edges are the distinct vertex
 *       pairs of the tets).  A vertex DoF is Dirichlet as its vertex; an edge
 *       DoF when the edge lies on a boundary face (a face of one tet only)
 *       whose three vertices are Dirichlet.  An edge DoF belongs to the
 *       partition id of its lower vertex if that id owns a non-Dirichlet
 *       vertex, else to that of its upper vertex.  Subdomains grow by delta
 *       (>= 1) element layers over the vertices as for P1 and hold the vertex
 *       DoFs and the edge DoFs with both ends inside.  The transfers are the
 *       P2 interpolation (the coarse P2 basis evaluated at the fine DoF
 *       points; restriction by its transpose).  Loads: MSP_F_ONE only
 *       (b_i = integral of phi_i).
 *   MSP_PDE_P2P1: two fields of different element order on one mesh, a P2
 *       field u (vertices and edges) and a P1 field p (vertices), coupled:
 *       -div(k grad u) + sigma k (u - p) = 1, -div(k grad p) + sigma k (p - u) = 1,
 *       sigma = msp_options.coupling > 0 (symmetric positive definite with the
 *       Dirichlet rows); N = (2,1,0,0).  DoF order: vertex 0's u, vertex 0's p,
 *       the u DoFs of its edges (0, b), b > 0 ascending, vertex 1's u, its p,
 *       ...; a p DoF is Dirichlet and belongs to a partition as its vertex;
 *       subdomains hold both fields of their vertices.  The transfers are split
 *       by field (Section 2.1, I = sum_f R_f^T I_f R~_f): the P2 interpolation
 *       on the u DoFs, the P1 barycentric one on the p DoFs.  Loads: MSP_F_ONE
 *       (f = 1 for both fields). */
typedef enum msp_pde {
  MSP_PDE_POISSON = 0, MSP_PDE_ELASTICITY = 1, MSP_PDE_POISSON_P2 = 2, MSP_PDE_P2P1 = 3
} msp_pde;

/* One mesh level (Section 2.1: the mesh perspective M = (K, N); the DoFs
 * per vertex follow msp_options.pde).  All arrays are host memory, copied. */
typedef struct msp_level_desc {
  int32_t n_nodes;            /* number of vertices (DoFs: n_nodes x fields) */
  const double* xyz;          /* [n_nodes][3] coordinates */
  int32_t n_tets;             /* number of tetrahedra */
  const int32_t* tets;        /* [n_tets][4] vertex ids, any orientation */
  const uint8_t* dirichlet;   /* [n_nodes] 1 = homogeneous Dirichlet node */
  const int32_t* owner;       /* [n_nodes] partition id of every vertex (Section 2.2:
                                 the non-overlapping subdomains); required on every
                                 level but the coarsest, and there too with
                                 MSP_COARSE_RAS (ignored with MSP_COARSE_DIRECT) */
} msp_level_desc;

typedef void* (*msp_alloc_fn)(void* ctx, size_t bytes, void* stream);
typedef void (*msp_free_fn)(void* ctx, void* ptr, void* stream);

/* Transfers between consecutive levels (msp_options.transfer). */
typedef enum msp_transfer {
  MSP_TRANSFER_BARY = 0,  /* P = barycentric interpolation of level-(l+1) fields at the
                             nodes of level l; restriction by P^T */
  MSP_TRANSFER_MLS = 1    /* overlapping moving-least-squares interpolation in both
                             directions (Section 3.2, Eq. 13-15, 24); see below */
} msp_transfer;

/* The coarsest level (msp_options.coarse_solver). */
typedef enum msp_coarse {
  MSP_COARSE_DIRECT = 0,  /* one interior block, factored and solved exactly (FP64) */
  MSP_COARSE_RAS = 1      /* RAS-smoothed like the other levels, as Algorithm 2 states:
                             nu_pre steps from z = 0; the level then needs an owner
                             array.  With nlevels == 1 and nu_pre == 1 the preconditioner
                             is one-level RAS (Eq. 7). */
} msp_coarse;

typedef struct msp_options {
  int32_t delta;              /* overlap: element layers added to each subdomain (>= 0) */
  int32_t nu_pre, nu_post;    /* RAS smoothing steps before / after the coarse correction */
  int32_t restart;            /* FGMRES restart length m (1..256) */
  int32_t max_it;             /* FGMRES iteration cap */
  int32_t factor_precision;   /* msp_precision */
  int32_t coef_kind;          /* msp_coef */
  int32_t wave[8][3];         /* a_j for MSP_K_COSEXP */
  double coef_scale;          /* s for MSP_K_COSEXP */
  int32_t load_kind;          /* msp_load */
  int32_t transfer;           /* msp_transfer */
  int32_t restrict_scaling;   /* MSP_TRANSFER_MLS only.  1 (default): the residual is
                                 restricted as a density, r_i / |w_i| (|w_i| = sum of |T|/4
                                 over the tets at node i), and the result multiplied by the
                                 coarse |w|, so that its scale matches the coarse operator;
                                 0: the plain interpolated residual of Algorithm 2 */
  int32_t coarse_solver;      /* msp_coarse */
  int32_t ilu_fill_fine;      /* subdomain solver of level 0: -1 (default) the exact LU of the
                                 block (dense tile envelope); p >= 0 ILU(p), the incomplete LU
                                 with the level-of-fill pattern (Section 4.4 uses ILU(2)) */
  int32_t ilu_fill_coarse;    /* the same for the smoothed levels 1.. (Section 4.4: ILU(0)).
                                 ILU levels factor and sweep in FP64 with MSP_F64, in FP32
                                 with MSP_F32 or MSP_BF16; the coarsest level stays direct */
  int32_t pde;                /* msp_pde (default MSP_PDE_POISSON) */
  double poisson_ratio;       /* MSP_PDE_ELASTICITY: in (0, 0.5), default 0.3; the transfers
                                 must then be MSP_TRANSFER_BARY */
  double coupling;            /* MSP_PDE_P2P1: the coupling coefficient sigma > 0, default 1 */
  int32_t host_only;          /* 1: build the host-side structures only (no device use);
                                 only msp_hierarchy_copy / info work on such a handle */
  size_t mem_budget_bytes;    /* 0 = unlimited; instances beyond it get MSP_ERR_OOM */
  msp_alloc_fn alloc;         /* optional device allocator (NULL: cudaMalloc) */
  msp_free_fn free;
  void* alloc_ctx;
} msp_options;

/* Fills *o with the defaults: delta 1, nu 2/2, restart 30, max_it 1000, FP64
 * factors, k = 1, f = 1, barycentric transfers (MLS restriction scaling on),
 * direct coarsest solve, exact subdomain LU (no ILU), no budget, cudaMalloc. */
MSP_API void msp_default_options(msp_options* o);

typedef struct msp_hierarchy msp_hierarchy;
typedef struct msp_instance msp_instance;

typedef struct msp_stats {
  int32_t status;             /* msp_status of the call */
  int32_t iterations;         /* FGMRES iterations (V-cycles) */
  double rel_residual;        /* ||b - A x|| / ||b||, true residual, FP64 */
  double ms_assemble, ms_factor, ms_solve;  /* host wall time of each stage */
  double ms_queue, ms_total;  /* msp_poll only: time queued, and submit-to-done */
} msp_stats;

/* ---- set-up, once per hierarchy (Algorithm 2, lines "construct the hierarchy
 * and provide J per level"; reuse across parameters, Sections 1 and 4.1) ----
 * lv[0..nlevels-1], finest first, nlevels >= 1.  Builds on the host: the CSR
 * pattern of every level, the element-to-nonzero contribution map, the
 * delta-overlapping subdomains (Section 2.2), the dense-block extraction maps,
 * and the transfers: with MSP_TRANSFER_BARY point location and the barycentric
 * interpolation P (coarse l+1 -> fine l) with its transpose; with
 * MSP_TRANSFER_MLS the two MLS operators of Section 3.2.  MLS row at a target
 * node x* owned by id q: the source nodes of Omega^delta_q (source vertices
 * owned by q, Dirichlet ones included, grown by delta element layers) within
 * rho of x*, weights w = 1 - 6s^2 + 8s^3 - 3s^4 (s = distance / rho, Eq. 15),
 * row = p(x*)^T P1^{-1} P2 for the linear basis; rho = c h with h =
 * cbrt(6 |bounding box| / tets) of level l+1 and c = 1.5, 1.5^2, ... until the
 * neighbourhood has rank 4 (Theorem 3.2).  Subdomain q of one level is
 * subdomain q of the other when both levels are partitioned over the same id
 * set; otherwise (and for the coarsest level) the neighbourhood comes from the
 * whole source level.  Dirichlet source nodes take part in the fit and are
 * then dropped as columns; Dirichlet target nodes get empty rows.  Then it
 * uploads everything and computes the per-tet geometry and the load vector on
 * the device.  Errors: MSP_ERR_INVALID (degenerate tet, index out of range,
 * missing owner array, bad option, an MLS neighbourhood that never reaches
 * rank 4), MSP_ERR_OOM. */
MSP_API int msp_load_hierarchy(const msp_level_desc* lv, int nlevels, const msp_options* o,
                       msp_hierarchy** out);
MSP_API void msp_free_hierarchy(msp_hierarchy* h);

/* Sizes of level `level`: n_nodes, nnz, number of subdomains (0 on the
 * coarsest level), sum over subdomains of n_p (DoFs), and factor elements.
 * Vectors of a level (msp_apply, msp_solve, ...) hold n_dofs entries. */
typedef struct msp_level_info {
  int32_t n_nodes, n_tets;    /* vertices and tetrahedra */
  int64_t nnz;
  int32_t n_sub;
  int64_t sub_dofs;           /* sum_p n_p (coarsest: interior DoFs) */
  int64_t factor_elems;       /* elements of the tiled factor storage of this level */
  int64_t P_nnz;              /* nnz of P from level+1 (0 on the coarsest) */
  int64_t R_nnz;              /* nnz of the restriction to level+1 (P^T or MLS) */
  int32_t fac_ctas;           /* CTAs of the one persistent factorisation launch of this level
                                 (0: tile-step launches, or a host-only hierarchy) */
  int32_t ras_ctas;           /* CTAs of the staged RAS solve (0: directly solved level) */
  int32_t spmv_lanes[3];      /* lanes per row of the SpMV schedules picked at load time by
                                 timing them on the device: 2/4/8/16/32, 1 (one lane per row
                                 over row blocks staged in shared memory), or 64 (one thread per
                                 row of the four-entry form of an operator with at most four
                                 entries per row: the barycentric P); J, prolongation,
                                 restriction (0: host-only hierarchy or no such operator).
                                 The environment variable MSP_SPMV_LANES = 1, 2, 4, 8, 16, 32 or
                                 64, read at load time, fixes the schedule instead (where it
                                 applies) */
  int32_t n_dofs;             /* DoFs: n_nodes x fields per vertex (msp_options.pde) */
} msp_level_info;
MSP_API int msp_hierarchy_info(const msp_hierarchy* h, int level, msp_level_info* info);

/* ---- per parameter (Eq. 2-4 on every level) ----
 * Creates an instance bound to `stream` and assembles J(mu) (CSR values) on
 * every level.  mu: host array of n_mu doubles (n_mu == 8 for MSP_K_COSEXP,
 * ignored for MSP_K_CONST).  Errors: MSP_ERR_INVALID (non-finite mu, wrong
 * n_mu), MSP_ERR_OOM (allocation or budget). */
MSP_API int msp_assemble(msp_hierarchy* h, const double* mu, int n_mu, void* stream,
                 msp_instance** out);
/* Re-assembles an existing instance for a new mu (no allocation). */
MSP_API int msp_reassemble(msp_instance* inst, const double* mu, int n_mu);
MSP_API void msp_free_instance(msp_instance* inst);

/* Subdomain blocks J^delta_p = R J R^T of every smoothed level (Eq. 6) and
 * their unpivoted LU factors in symmetric form (unit lower L, D; U = D L^T),
 * plus the FP64 factor of the coarsest level's interior block. */
MSP_API int msp_factor(msp_instance* inst);

/* msp_factor of n instances at once (Eq. 6 for every block of every
 * instance), for batches of parameters, possibly on hierarchies of different
 * sizes.  The blocks of every level that msp_factor factors in one persistent
 * launch (levels with many blocks) go into ONE persistent launch for the whole
 * batch per factor type, balanced longest-first over the GPU; the other
 * levels (the coarsest block's tile steps) run per instance on the
 * instance's own streams, concurrently.  Each block's arithmetic is that of
 * msp_factor, so the factors are bitwise the same.  insts: n distinct
 * assembled instances (host array, not kept); stream: the stream of the
 * batched launch (NULL: the first instance's), ordered after every
 * instance's assembly; every instance's stream is ordered after the batch,
 * and the call synchronises them all.  The launch's work lists are allocated
 * and freed inside the call.  Errors: MSP_ERR_INVALID (no instances, one
 * not assembled or listed twice, BF16 factors or ILU levels), MSP_ERR_OOM,
 * MSP_ERR_CUDA, MSP_ERR_INTERNAL (a pivot; the instance stays unfactored).
 * The profiling counters do not include the batched launch. */
MSP_API int msp_factor_batch(msp_instance* const* insts, int n, void* stream);

/* ---- batched solves: several instances, shared launches ----
 * A batch groups up to 32 factored instances (of one hierarchy or of several,
 * e.g. parameters of a family on meshes of different sizes) whose FGMRES
 * solves then run in lockstep with their launches fused: per level depth one
 * staged RAS launch over the blocks of every member (per factor type), one
 * SpMV launch per operator and schedule over the members' stacked rows, one
 * coarsest-solve launch with a cluster per member, one launch per Krylov
 * kernel, and one host synchronisation per iteration for the whole batch.
 * Each member's arithmetic is exactly that of its own msp_solve (the same
 * per-row, per-block and per-slice code in the same order), so its solution,
 * iterations and residual are bitwise those of msp_solve.
 *
 * msp_batch_create: insts holds n distinct instances (host array, copied; the
 * instances must outlive the batch and keep their factor storage, i.e. stay
 * allocated).  All members need the same nu_pre / nu_post, the directly
 * solved coarsest level and the exact subdomain LU (no ILU(p) levels); any
 * factor precision, also mixed within a batch.  stream: the stream the
 * batched work runs on (NULL: the first member's).  The call allocates the
 * fused launches' work lists (device memory, through the members'
 * allocator) and builds them on the host.  Errors: MSP_ERR_INVALID (n
 * outside 1..32, NULL or repeated members, members that differ as above or
 * live on different devices), MSP_ERR_OOM, MSP_ERR_CUDA.
 *
 * msp_solve_batch: FGMRES (as msp_solve) for every member at once, member i
 * solving J_i x_i = b_i with b_dev[i] (device, or NULL entries / a NULL
 * array for the assembled load vectors) into x_dev[i] (device).  Every member
 * must be factored (msp_factor or msp_factor_batch after its last
 * re-assembly).  The batch stream waits for each member's stream first, and
 * each member's stream waits for the batch at the end; the call synchronises
 * the batch stream.  st: NULL or n msp_stats, filled per member (ms_solve is
 * the batch's wall time).  Returns MSP_OK when every member converged, else
 * the first failing member's status (MSP_ERR_TIMEOUT for an expired bounded
 * wait first, MSP_ERR_NOT_CONVERGED, ...); the per-member statuses are in st. */
typedef struct msp_batch msp_batch;
MSP_API int msp_batch_create(msp_instance* const* insts, int n, void* stream, msp_batch** out);
MSP_API void msp_batch_free(msp_batch* b);
/* msp_batch_assemble: msp_reassemble of every member (Eq. 2-4 for its mu),
 * member i's parameters at mu[i * n_mu .. (i+1) * n_mu) (host), each on its own
 * stream, one synchronisation for all.  Errors as msp_reassemble. */
MSP_API int msp_batch_assemble(msp_batch* b, const double* mu, int n_mu);
/* msp_batch_factor: msp_factor of every member (Eq. 6), with the blocks of the
 * persistent levels of every FP64 / FP32 member in ONE persistent launch per
 * factor type over the batch (longest blocks first, on all SMs but a few that
 * the members' coarsest-block tile steps keep), the other levels on each
 * member's own streams concurrently.  Each block's arithmetic is that of
 * msp_factor, so the factors are bitwise the same.  From the second call on,
 * the whole batched factorisation replays from one CUDA graph.  Synchronises
 * the batch stream.  Errors: MSP_ERR_INVALID (a member not assembled),
 * MSP_ERR_INTERNAL (a pivot; that member stays unfactored), MSP_ERR_TIMEOUT,
 * MSP_ERR_CUDA. */
MSP_API int msp_batch_factor(msp_batch* b);
MSP_API int msp_solve_batch(msp_batch* b, const double* const* b_dev, double* const* x_dev, double rtol,
                            msp_stats* st);

/* One application of the V-cycle preconditioner of Algorithm 2 (z = B^{-1} r)
 * with the fine->coarse transfer P^T, coarse->fine P and a direct coarsest
 * solve.  r_dev, z_dev: device arrays of n_dofs(level 0) doubles; they must
 * not overlap.  Requires msp_factor. */
MSP_API int msp_apply(msp_instance* inst, const double* r_dev, double* z_dev, void* stream);

/* Right-preconditioned FGMRES(restart) on J(mu) x = b (Eq. 5), x_0 = 0,
 * stopping when ||b - J x|| <= rtol ||b|| (true residual).  b_dev: device
 * right-hand side, or NULL for the assembled load vector.  x_dev: device
 * output.  Synchronises the instance stream.  MSP_ERR_NOT_CONVERGED leaves the
 * last iterate in x_dev. */
MSP_API int msp_solve(msp_instance* inst, const double* b_dev, double* x_dev, double rtol,
              msp_stats* st);

/* The whole per-parameter path from host memory: re-assemble for mu, factor,
 * solve, copy the solution back.  b_host: NULL for the load vector, else
 * n_dofs doubles; x_host: n_dofs doubles. */
MSP_API int msp_solve_host(msp_instance* inst, const double* mu, int n_mu, const double* b_host,
                   double* x_host, double rtol, msp_stats* st);

/* Device bytes one instance of `h` needs (CSR values, factors, level vectors,
 * Krylov basis), for admission decisions. */
MSP_API int msp_instance_bytes(const msp_hierarchy* h, size_t* bytes);

/* ---- serving: continuous batching over resident hierarchies ----
 * A server owns worker slots.  Each slot is one instance of one hierarchy
 * with its own CUDA stream and host thread, running the whole per-parameter
 * path (assemble, factor, FGMRES, copy back) for one request at a time.
 * Slots are created on demand, up to slots_per_hierarchy per hierarchy, and
 * only while the server's device-memory budget has room for another instance
 * (admission by memory).  Requests that arrive while others are running go to
 * any idle slot of their hierarchy at once, so their device work overlaps;
 * otherwise they wait in a FIFO queue per hierarchy.  Every slot computes with
 * fixed-order reductions, so a request's result does not depend on what else
 * is running.  The caller keeps ownership of the hierarchies, which must
 * outlive the server. */
typedef struct msp_server msp_server;
typedef struct msp_server_opts {
  int32_t slots_per_hierarchy;  /* >= 1 */
  size_t mem_budget_bytes;      /* device bytes for all slots' instances; 0 = unlimited */
  double rtol_default;          /* used when msp_submit gets rtol <= 0 */
} msp_server_opts;
MSP_API void msp_server_default_options(msp_server_opts* o);
MSP_API int msp_server_create(const msp_server_opts* o, msp_server** out);
/* Registers a device-resident hierarchy; *id receives its handle (0, 1, ...). */
MSP_API int msp_server_add_hierarchy(msp_server* srv, msp_hierarchy* h, int* id);
/* Queues one solve of hierarchy `hierarchy_id` for parameter mu (host array,
 * copied) to relative residual rtol with the hierarchy's load vector as
 * right-hand side.  *req_id receives the request handle.  MSP_ERR_INVALID for
 * a bad id or mu; MSP_ERR_OOM if the budget cannot hold even one instance of
 * the hierarchy. */
MSP_API int msp_submit(msp_server* srv, int hierarchy_id, const double* mu, int n_mu, double rtol,
                       uint64_t* req_id);
/* Waits up to timeout_ms (0: no wait, < 0: no limit) for a request.
 * Returns MSP_PENDING if it has not finished (the request stays queued);
 * otherwise the request's own status, copies the solution (n_dofs of level
 * 0) into x_host when non-NULL, fills *st (ms_queue / ms_total included) and
 * forgets the request.  MSP_ERR_INVALID for an unknown req_id. */
MSP_API int msp_poll(msp_server* srv, uint64_t req_id, double* x_host, msp_stats* st, int timeout_ms);
/* Stops the workers after their current request, frees every slot. */
MSP_API void msp_server_free(msp_server* srv);

/* ---- single operators of the path, for parity checks and composition ----
 * y = op(x) on level `level`, device arrays, enqueued on `stream`:
 *   MSP_OP_SPMV     y = J_l x                     (n_l -> n_l)
 *   MSP_OP_RESIDUAL y = y - J_l x  (y holds r on entry)
 *   MSP_OP_INTERP   y = P_l x      (n_{l+1} -> n_l), l < L-1
 *   MSP_OP_RESTRICT y = P_l^T x    (n_l -> n_{l+1}), l < L-1
 *   MSP_OP_RAS      y = B_l^{-1} x (Eq. 7), l < L-1, needs msp_factor
 *   MSP_OP_COARSE   y = J_{L-1}^{-1} x, l = L-1, needs msp_factor */
typedef enum msp_op {
  MSP_OP_SPMV = 0, MSP_OP_RESIDUAL = 1, MSP_OP_INTERP = 2, MSP_OP_RESTRICT = 3,
  MSP_OP_RAS = 4, MSP_OP_COARSE = 5
} msp_op;
MSP_API int msp_apply_op(msp_instance* inst, int op, int level, const double* x_dev, double* y_dev,
                 void* stream);

/* ---- introspection: copy a named array into host memory ----
 * Hierarchy arrays (index structures, host-resident):
 *   MSP_ARR_ROWPTR, MSP_ARR_COL (int32), MSP_ARR_SUB_PTR, MSP_ARR_SUB_DOFS (int32),
 *   MSP_ARR_SUB_NT (int32 tiles per side of each block), MSP_ARR_TILE_FIRST (int32
 *   F_I of every tile row, blocks concatenated; see MSP_TILE),
 *   MSP_ARR_SUB_OWN (uint8), MSP_ARR_P_ROWPTR, MSP_ARR_P_COL (int32),
 *   MSP_ARR_P_VAL (double) of the prolongation from level+1 (P or MLS),
 *   MSP_ARR_PT_ROWPTR, MSP_ARR_PT_COL (int32), MSP_ARR_PT_VAL (double) of the
 *   restriction to level+1 (P^T or MLS), MSP_ARR_LOAD (double, device-resident b)
 * Instance arrays (device-resident, copied back):
 *   MSP_ARR_VAL (double CSR values), MSP_ARR_FACTOR (the tiled factor of
 *   subdomain `sub` of `level`, sub = -1 for the coarsest level, in the
 *   precision of that level's factors).
 * ILU(p) levels (msp_options.ilu_fill_*): MSP_ARR_ILU_PTR (int64, rows + 1)
 *   and MSP_ARR_ILU_COL (int32 local columns) give the strict lower pattern
 *   of every block, row R = sub_ptr[p] + i for local row i of subdomain p;
 *   MSP_ARR_ILU_VAL (the unit lower L on that pattern) and MSP_ARR_ILU_D
 *   (one per row) are the instance's factors, U = D L^T: double with
 *   MSP_F64, float with MSP_F32 or MSP_BF16 (ILU levels are never BF16).
 * bytes_out receives the array size; with dst == NULL only the size is
 * returned.  MSP_ERR_INVALID if cap is too small. */
typedef enum msp_array {
  MSP_ARR_ROWPTR = 0, MSP_ARR_COL = 1, MSP_ARR_SUB_PTR = 2, MSP_ARR_SUB_DOFS = 3,
  MSP_ARR_SUB_OWN = 4, MSP_ARR_P_ROWPTR = 5, MSP_ARR_P_COL = 6, MSP_ARR_P_VAL = 7,
  MSP_ARR_PT_ROWPTR = 8, MSP_ARR_PT_COL = 9, MSP_ARR_PT_VAL = 10, MSP_ARR_LOAD = 11,
  MSP_ARR_VAL = 12, MSP_ARR_FACTOR = 13, MSP_ARR_SUB_NT = 14, MSP_ARR_TILE_FIRST = 15,
  MSP_ARR_ILU_PTR = 16, MSP_ARR_ILU_COL = 17, MSP_ARR_ILU_VAL = 18, MSP_ARR_ILU_D = 19
} msp_array;
MSP_API int msp_hierarchy_copy(const msp_hierarchy* h, int level, int what, void* dst, size_t cap,
                       size_t* bytes_out);
MSP_API int msp_instance_copy(const msp_instance* inst, int level, int what, int sub, void* dst,
                      size_t cap, size_t* bytes_out);

/* Tile edge of the factor storage.  Every block of n_p DoFs (ascending global
 * ids) is padded to NT = ceil(n_p / 64) tiles per side (the padding is an
 * identity block).  Only its tile envelope is stored: tile row I holds the
 * tiles (I, F_I) .. (I, I), 64 x 64 row-major each, rows one after another,
 * where F_I (nondecreasing) is the first tile column with a nonzero in tile
 * rows >= I.  Without pivoting the factors stay inside that envelope.  In a
 * diagonal tile the strict lower part holds L, the diagonal holds D and the
 * strict upper part holds the transpose of the inverse of the unit lower
 * diagonal block of L. */
#define MSP_TILE 64

/* ---- per-kernel accounting ----
 * Every launch is counted per kernel class with its algorithmic bytes and
 * flops (bytes the operation must move at least once, flops it must do).
 * Classes in `class_mask` (bit = 1 << class) are also timed with CUDA events
 * recorded around each launch on the launching stream. */
typedef enum msp_kernel_class {
  MSP_PK_ASSEMBLE = 0,     /* coefficient + assembly of J(mu), every level */
  MSP_PK_EXTRACT = 1,      /* dense subdomain blocks from CSR; BF16 rounding of the factors */
  MSP_PK_LDLT_DIAG = 2,    /* diagonal tile factorisation */
  MSP_PK_LDLT_PANEL = 3,   /* panel solves */
  MSP_PK_LDLT_TRAIL = 4,   /* trailing (Schur complement) updates */
  MSP_PK_RAS = 5,          /* RAS application on level 0 */
  MSP_PK_RAS_COARSER = 6,  /* RAS application on levels 1..L-2 */
  MSP_PK_COARSE = 7,       /* coarsest-level direct solve */
  MSP_PK_SPMV = 8,         /* J x and residuals */
  MSP_PK_TRANSFER = 9,     /* P and P^T */
  MSP_PK_VEC = 10,         /* Krylov dots, axpys, copies */
  MSP_PK_LDLT_BLOCKS = 11, /* whole-block factorisation, one persistent launch per level */
  MSP_PK_COUNT = 12
} msp_kernel_class;

typedef struct msp_kernel_profile {
  int64_t launches;        /* kernels launched */
  double bytes;            /* algorithmic bytes of those launches */
  double flops;            /* algorithmic flops of those launches */
  int64_t timed;           /* launches covered by ms */
  double ms;               /* summed CUDA-event duration of the timed launches */
} msp_kernel_profile;

MSP_API int msp_profile_enable(msp_instance* inst, uint32_t class_mask);
MSP_API int msp_profile_reset(msp_instance* inst);
MSP_API int msp_profile_read(msp_instance* inst, int kclass, msp_kernel_profile* out);

/* ---- failure injection on the host, for tests (no counterpart in the paper) ----
 * The next `count` staged RAS applications of this instance (the smoothed
 * levels' triangular solves, Eq. 7) are launched with no tile copies issued:
 * every bounded wait of those launches on a tile that never arrives runs out
 * after a short limit, their output is meaningless, and the expiry is
 * recorded.  No copy is ever in flight and nothing else changes, so the
 * context stays usable and later calls work normally; msp_solve (and
 * msp_solve_host) then return MSP_ERR_TIMEOUT, which takes precedence over
 * the iteration's own status, and clear the record.  count = 0 cancels.
 * Errors: MSP_ERR_INVALID (NULL instance, count < 0). */
MSP_API int msp_debug_expire_waits(msp_instance* inst, int count);

/* ---- work placement, for tests (no counterpart in the paper) ----
 * The persistent FP64 factorisation and the staged RAS solves split their
 * blocks into work lists per SM, and a CTA takes the list of the SM it runs
 * on (read on the device); lists that no CTA of their SM takes (an SM the
 * launch does not reach, or a CTA beyond its SM's share) are taken by other
 * CTAs.  With bit 0 of `on` set this instance's launches use twice as many
 * lists as SMs, so that half of the lists are always taken that way; the
 * blocks' arithmetic does not depend on which CTA takes them, so factors and
 * solutions are bitwise those of on == 0.  A factorisation graph captured
 * before the switch is dropped (the call waits for the instance's stream).
 * Bit 1: the coarsest level's cluster solve takes its 8-CTA form, the one it
 * falls back to where the GPU cannot place a cluster of 16 (the same sweeps
 * over 8 rows a CTA; sums in another order, so equal to rounding).
 * Errors: MSP_ERR_INVALID (NULL instance), MSP_ERR_CUDA. */
MSP_API int msp_debug_spread_work(msp_instance* inst, int on);

/* ---- tensor-core self-check (no counterpart in the paper) ----
 * Multiplies two fixed 128 x 64 BF16 matrices with integer entries on the
 * current device through the library's tcgen05 path (operands in shared
 * memory, FP32 accumulators in tensor memory) and compares every one of the
 * 128 x 128 results bit for bit with the exact integer product computed on
 * the host.  *mismatches (may be NULL) receives the number of differing
 * entries.  Returns MSP_OK, MSP_ERR_INTERNAL (a mismatch), MSP_ERR_TIMEOUT
 * (the bounded wait for the MMA expired), MSP_ERR_CUDA or MSP_ERR_OOM. */
MSP_API int msp_tensor_selftest(int* mismatches);

/* ---- allocation-free multi-vector dot product ----
 * No counterpart in the paper: a library convenience for callers that may not
 * allocate device memory when they need the result (code under a memory
 * manager that owns all device memory and forbids further allocations,
 * real-time loops that cannot risk an allocation stalling or failing).
 * out_dev[i] = sum_{k<n} V_dev[i*ld + k] * w_dev[k] for i < nv, computed by
 * the same kernels and fixed-order two-stage reduction FGMRES uses for its
 * Gram-Schmidt coefficients and norms, so results are bitwise those of the
 * solver's reduction and bitwise reproducible.  All pointers are
 * caller-owned device memory on the current device; `stream` as above.  The
 * partial sums live in one fixed device array of MSP_NOALLOC_MAX_VECTORS x
 * 296 doubles (148 KiB) that every GPU loading the library holds until exit;
 * the call allocates nothing.  The first call on a device looks up that
 * array's device address with the device current and keeps it (make that
 * first call before any stream capture; after cudaDeviceReset of a device
 * the kept address is stale, so do not call it on that device again).  Every
 * call reuses the array, so calls that overlap on the GPU race; each call
 * overwrites every entry it reads, so nothing needs clearing.  Errors:
 * MSP_ERR_INVALID for nv outside 1..MSP_NOALLOC_MAX_VECTORS, n < 0, ld < n
 * (nv > 1) or NULL pointers; MSP_ERR_CUDA if the launch fails. */
#define MSP_NOALLOC_MAX_VECTORS 64
MSP_API int msp_multidot_noalloc(const double* V_dev, int64_t ld, int nv, const double* w_dev,
                                 int64_t n, double* out_dev, void* stream);

/* Thread-local message of the last failed call on this thread ("" if none). */
MSP_API const char* msp_last_error(void);
/* Library version string. */
MSP_API const char* msp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MSP_H_ */
