/*
 * hz.h — C ABI of the GB300 two-level ORAS / FGMRES Helmholtz solver.
 *
 * The library solves the Galerkin P3 discretisation (Lagrange elements of
 * order 3 on a tetrahedral mesh) of the acoustic Helmholtz equation,
 * Sec. "Tetrahedral finite element method", Eq. eqh and Eq. eq1:
 *
 *     -Lap u - k^2 u = s  in Omega,   k = omega / c(x),  omega = 2 pi f,
 *     d_n u - i k u = g   on absorbing (Robin) faces,
 *     u = 0               on Dirichlet (free-surface) faces,
 *
 * (time convention e^{-i omega t}; a unit point source radiates like
 * e^{ikr} / (4 pi r)), i.e. the complex-symmetric sparse system
 *     A = sum_e (K_e - omega^2 m_e M_e) - i omega sum_{Robin f} sqrt(m_e) B_f,
 * m_e = 1 / c_e^2, by flexible GMRES (Sec. "Domain decomposition
 * preconditioner") preconditioned by the two-level method of Eq. 2lvl,
 *     M^{-1} = M1^{-1} (I - A Q) + Q,  Q = Z E^{-1} Z^T,  E = Z^T A Z,
 * with the one-level optimized restricted additive Schwarz operator of
 * Eq. oras, M1^{-1} = sum_i R_i^T D_i A_i^{-1} R_i, whose local matrices A_i
 * carry absorbing conditions on the subdomain interfaces. The coarse problem
 * is solved by a fixed number of GMRES iterations preconditioned by one-level
 * ORAS on the coarse mesh (10 in the paper).
 *
 * Conventions for every call:
 *   - Units: metres, m/s, Hz. Complex numbers are interleaved (re, im)
 *     doubles, the layout of a C99 double complex / torch.complex128.
 *   - Blocks of right-hand sides and wavefields are source-major:
 *     [ns][n][2] doubles (each source's n complex values contiguous).
 *   - Dof numbering is the library's own; hz_dof_coords gives the node
 *     coordinates so that callers can match dofs by position.
 *   - Input arrays are read during the call and stay owned by the caller;
 *     output arrays are caller-allocated. A context owns all the device
 *     memory it allocates until hz_free.
 *   - The library runs its kernels on a stream of its own; every call first
 *     waits for the work already queued on the CUDA stream given to
 *     hz_setup and returns after its own work has completed. A context is
 *     not thread-safe; one call at a time per context.
 *   - Every int-returning call returns HZ_OK (0) or an HZ_E* code and never
 *     aborts; hz_last_error() gives a one-line description of the last error
 *     on the calling thread.
 */
#ifndef HZ_H
#define HZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HZ_OK = 0,
  HZ_EINVAL = 1,      /* bad mesh, partition, size or option */
  HZ_ENOMEM = 2,      /* device or host allocation failed */
  HZ_ECUDA = 3,       /* a CUDA runtime call failed */
  HZ_EINTERNAL = 4,   /* inconsistent internal state (a bug) */
  HZ_ESINGULAR = 5,   /* zero pivot with perturbation disabled (pivot_tau = 0) */
  HZ_ENOTCONV = 6,    /* maxit reached; outputs hold the last iterate */
  HZ_EBREAKDOWN = 7   /* Krylov breakdown that left a column unconverged */
};

enum { HZ_BC_ROBIN = 0, HZ_BC_DIRICHLET = 1 };
enum { HZ_COARSE_NONE = 0, HZ_COARSE_GMRES = 1, HZ_COARSE_DIRECT = 2 };
enum { HZ_PREC_FP64 = 0, HZ_PREC_MIXED = 1 };

typedef struct hz_ctx hz_ctx; /* opaque */

/* Tetrahedral mesh. Boundary faces not listed in bfaces get the natural
 * (homogeneous Neumann) condition; a listed face must be exterior. */
typedef struct hz_mesh {
  const double* xyz;        /* [nv][3] vertex coordinates, metres */
  int64_t nv;
  const int32_t* tets;      /* [ne][4] vertex ids in [0, nv) */
  int64_t ne;
  const int32_t* bfaces;    /* [nbf][3] vertex ids of exterior triangles */
  const int32_t* bface_tag; /* [nbf] HZ_BC_ROBIN (absorbing) or HZ_BC_DIRICHLET (free surface) */
  int64_t nbf;
} hz_mesh;

typedef struct hz_options {
  int32_t precision;        /* HZ_PREC_FP64 (default) or HZ_PREC_MIXED */
  double rtol;              /* FGMRES stop: ||b - A u|| / ||b|| <= rtol per column (1e-6) */
  int32_t maxit;            /* maximum FGMRES iterations (500) */
  int32_t restart;          /* FGMRES restart length m (30) */
  int32_t max_block;        /* maximum right-hand sides per block (64) */
  int32_t coarse_mode;      /* HZ_COARSE_GMRES (default), HZ_COARSE_NONE, HZ_COARSE_DIRECT */
  int32_t coarse_inner_its; /* inner coarse GMRES iterations (10) */
  int32_t leaf_size;        /* nested-dissection leaf size (64) */
  double pivot_tau;         /* static pivot perturbation, relative to max|A_i| (1e-12; an FP32 factorisation
                               uses at least 1e-6); 0 disables it (a zero pivot is then HZ_ESINGULAR) */
  int32_t verbose;          /* 0 silent */
  int32_t use_graphs;       /* 1 (default): replay the local-solve and coarse-solve launch sequences
                               as captured CUDA graphs; 0: launch them one by one */
  int32_t tensor_cores;     /* mixed form only. 1: front-sweep tiles of at least 32 rows and 32 reduction
                               indices run on the tcgen05 tensor cores for blocks of 9-16 columns, as a
                               three-term TF32 split of the FP32 factors and inputs (hi*hi + hi*lo + lo*hi,
                               FP32 accumulation in TMEM), which keeps FP32 accuracy; other tiles and
                               block widths use the SIMT FP32 sweeps. 0: SIMT FP32 sweeps only */
  int32_t overlap;          /* element layers added around each subdomain, each layer = every element
                               sharing a vertex with the current set (1, the default; >= 1) */
  int32_t coarse_fp32;      /* mixed form only. 0 (default): E = Z^T A Z, Z, Z^T and the inner coarse GMRES
                               run with FP64 accuracy (as FP32 pairs under emulate_fp64); the coarse fronts,
                               factorised in FP64 like all fronts, are applied
                               in complex FP32 like the fine ones. 1: the whole of M^{-1}, coarse level
                               included, runs on complex FP32 blocks */
  int32_t debug_bounds;     /* 1: after the factorisation, one device pass checks every index map of the
                               hot path (restriction, ownership, front rows, extend-add sources, tiles)
                               against its bounds; a violation fails hz_setup with HZ_EINTERNAL. 0 (default) */
  int32_t block_arnoldi;    /* 0 (default): one Krylov space per right-hand side (per-column CGS with a
                               selective second pass). 1: block FGMRES for hz_solve / hz_solve_rhs /
                               hz_fwi_gradient, one Krylov space shared by the block: block CGS2 and CholQR2
                               as tall-skinny FP64 products, linearly dependent right-hand sides deflated;
                               needs max_block <= 32. Servers keep one Krylov space per column */
  int32_t persistent_sweeps;/* 1: each SIMT front sweep is one launch over all tree levels (resident CTAs take
                               tiles in level order and wait for the fronts they depend on); 0 (default): one
                               launch per level. The tensor-core tiles keep one launch per level */
  int32_t factor_fp32;      /* mixed form only. 1 (default): the fine fronts are factorised (partial LDL^T and
                               partitioned inverse) in complex FP32; 0: in FP64, then rounded to FP32. The
                               coarse fronts are factorised in FP64 in both forms */
  int32_t recycle;          /* Krylov subspace recycling (deflated restarting across cycles and solves, in the
                               spirit of GCRO-DR; the paper's outlook on reusing Krylov information across
                               sources). k in [1, 16]: after every FGMRES cycle the k/2 harmonic Ritz vectors
                               of smallest magnitude of the slowest column's cycle join a space U of at most k
                               vectors, kept by the context for every later solve of the same operator; C = A U
                               is kept orthonormal, each cycle starts from x += U C^H r and its Arnoldi runs on
                               (I - C C^H) A M^{-1}. 0 (default): off. Needs per-column FGMRES (block_arnoldi 0)
                               and restart >= 2; servers do not recycle. Costs 6 k n complex FP64 of device memory */
  int32_t emulate_fp64;     /* mixed form only. 1 (default): the products with A (Krylov products, true
                               residuals, hz_apply_A), the Gram-Schmidt products, updates and norms of the
                               FGMRES iteration and, with the FP64 coarse level, the products with E, Z and
                               Z^T and the coarse Krylov iteration run in double-float arithmetic (the
                               Hessenberg matrix, rotations, least squares and solution update stay FP64):
                               each double is carried as a pair of FP32 numbers
                               (about 48 significant bits; Dekker's TwoProduct and Knuth's TwoSum), which
                               GB300 issues 64 times faster than FP64 fused multiply-adds. Relative error of
                               a row of m nonzeros about m 2^-48 of sum |a_ij x_j|; magnitudes from about
                               1e-31 to 1e38 keep that precision (smaller ones FP32 precision). With
                               block_arnoldi or recycle the outer Krylov iteration (not its products) stays in
                               native FP64. 0: native FP64. The FP64 form always uses native FP64 */
  int32_t coarse_leaf_size; /* nested-dissection leaf size of the coarse level's local problems; 0 (default):
                               the same as leaf_size. The coarse problems are small and their sweeps bound
                               by per-level latency, so fewer, larger leaves can pay there */
} hz_options;

typedef struct hz_stats {
  int32_t iterations;       /* FGMRES iterations of the last solve (max over columns) */
  int32_t restarts;
  int32_t converged;        /* 1 if every column reached rtol (true residual) */
  int32_t ncols;
  double max_rel_residual;  /* max over columns of ||b - A u|| / ||b|| (true residual) */
  double solve_seconds;     /* wall time of the solve call */
  double setup_seconds;     /* wall time of hz_setup (host + device) */
  double factor_seconds;    /* device factorisation time inside hz_setup */
  int32_t perturbed_pivots; /* static pivot perturbations of the context's factorisations */
} hz_stats;

typedef struct hz_info {
  int64_t n;                /* global dofs */
  int64_t nnz;              /* nonzeros of A */
  int64_t nnz_imag;         /* entries of A with a nonzero imaginary part (Robin faces) */
  int32_t nparts;
  int64_t sub_rows;         /* sum of overlapping subdomain sizes n_i */
  int64_t n_coarse;         /* coarse dofs (0 without coarse level) */
  int64_t nnz_coarse;       /* nonzeros of E */
  int64_t factor_entries;   /* stored factor entries, fine level: sum_t k_t (k_t + 1)/2 + k_t m_t */
  int64_t coarse_factor_entries;
  int64_t front_entries;    /* sum_t f_t^2 (device front storage, fine level) */
  int32_t max_front;        /* largest front order f_t (fine) */
  int32_t nfronts;
  int32_t nlevels;          /* tree heights (fine) */
  int32_t perturbed_pivots; /* static perturbations applied in the factorisations */
  double device_bytes;      /* device memory held by the context */
  int64_t kernel_launches;  /* kernels launched by the library in this process so far (kernels of
                               replayed CUDA graphs included) */
  double factor_ldlt_seconds;    /* device time of the front assembly and partial LDL^T (both levels) */
  double factor_inverse_seconds; /* device time of the partitioned inverses (both levels) */
} hz_info;

/* Fills *opt with the defaults listed above. */
int hz_default_options(hz_options* opt);

/* Set up a solver for one mesh and frequency (Sec. "Domain decomposition
 * preconditioner"): P3 numbering, assembly of A, the overlapping subdomains
 * of the element partition (overlap: elements sharing a vertex), local Robin
 * matrices A_i, the coarse space on `coarse` (a mesh nested in `fine`, or
 * NULL for coarse_mode = HZ_COARSE_NONE), nested-dissection symbolic
 * analysis on the host and the batched multifrontal factorisation of every
 * A_i (and E_i / E) on the device.
 *   velocity  [ne] per-element wavespeed c_e > 0 (m/s)
 *   elem_part [ne] subdomain of each element, in [0, nparts); every part
 *             non-empty
 *   stream    cudaStream_t (NULL: the legacy default stream)
 * Errors: HZ_EINVAL (bad input), HZ_ENOMEM, HZ_ECUDA. *out is NULL on error. */
int hz_setup(const hz_mesh* fine, const double* velocity, double freq_hz, const int32_t* elem_part,
             int32_t nparts, const hz_mesh* coarse, const hz_options* opt, void* stream, hz_ctx** out);

int hz_ndof(const hz_ctx* ctx, int64_t* n);
/* Coordinates [n][3] of the P3 nodes in the library's dof order (host). */
int hz_dof_coords(const hz_ctx* ctx, double* xyz);
int hz_get_info(const hz_ctx* ctx, hz_info* info);

/* Wavefields for point sources (Sec. "Numerical results": a point source in
 * the subsurface): right-hand side F_j = a phi_j(x_s) in the lowest-index
 * element containing x_s, zero on Dirichlet dofs.
 *   src_xyz [ns][3], src_amp [ns][2] complex amplitudes
 *   u       [ns][n][2] output, host (u_on_device = 0) or device pointer
 *   stats   may be NULL
 * Blocks of up to max_block sources are solved together (one Krylov space
 * per source). Returns HZ_ENOTCONV when maxit is reached first (u then holds
 * the last iterate). */
int hz_solve(hz_ctx* ctx, const double* src_xyz, const double* src_amp, int32_t ns, double* u,
             int32_t u_on_device, hz_stats* stats);

/* Per-column results of the last hz_solve / hz_solve_rhs / hz_fwi_gradient call
 * on ctx, in source order (for hz_fwi_gradient: the forward solves, then the
 * adjoint ones): the true relative residual ||b - A u|| / ||b|| of each column
 * when the call returned, and the FGMRES iterations that column used (its own
 * accepted Arnoldi steps). rel_residual and iterations are caller-owned
 * arrays of cap entries (either may be NULL); *ncols receives the number of
 * columns of that call, which may exceed cap (only cap entries are written).
 * Errors: HZ_EINVAL. */
int hz_column_stats(const hz_ctx* ctx, double* rel_residual, int32_t* iterations, int32_t cap, int32_t* ncols);

/* Orthonormal basis of the last FGMRES restart cycle of the last solve
 * call (diagnostics and tests): *nblocks basis blocks of *ncols columns,
 * written to V [nblocks][ncols][n][2] (host, caller-owned, room for cap
 * blocks; only min(cap, *nblocks) are written). With block_arnoldi = 1 the
 * nblocks x ncols vectors are orthonormal together (deflated directions are
 * zero vectors); otherwise column c of every block belongs to the Krylov
 * space of right-hand side c alone. Errors: HZ_EINVAL (no solve yet), HZ_ECUDA. */
int hz_krylov_basis(hz_ctx* ctx, double* V, int32_t cap, int32_t* nblocks, int32_t* ncols);

/* Same for given right-hand sides F [ns][n][2] (host or device). */
int hz_solve_rhs(hz_ctx* ctx, const double* F, int32_t ns, int32_t F_on_device, double* u, int32_t u_on_device,
                 hz_stats* stats);

/* Y = A X, X and Y [s][n][2], host or device (both on the same side). */
int hz_apply_A(hz_ctx* ctx, const double* X, double* Y, int32_t s, int32_t on_device);

/* Y = M^{-1} X (Eq. 2lvl with the configured coarse mode; Eq. oras alone
 * with HZ_COARSE_NONE), X and Y [s][n][2]. */
int hz_apply_prec(hz_ctx* ctx, const double* X, double* Y, int32_t s, int32_t on_device);

/* Per-phase device timing of the hot path (CUDA events recorded around each
 * phase on the context's stream while profiling is on). Phases: "spmm_A"
 * (products with A), "fronts" (fine-level local solves), "restrict_prolong"
 * (fine R_i gathers and partition-of-unity scatters), "coarse" (Z^T, the
 * coarse solve and Z), "arnoldi" (outer orthogonalisation, least squares and
 * solution update), "precond_spmm" (the residual t = v - A q inside M^{-1},
 * FP32 in the mixed form). flops and bytes are the algorithmic counts of the
 * recorded calls (complex multiply-add = 8 flops; bytes = compulsory
 * traffic: matrix/factor entries, indices and the input/output blocks). */
typedef struct hz_phase_time {
  const char* name;
  int64_t calls;
  double ms;
  double flops;
  double bytes;
} hz_phase_time;

/* Reset the counters and start recording. */
int hz_profile_begin(hz_ctx* ctx);
/* Synchronise the stream, stop recording and write up to `cap` phases. */
int hz_profile_end(hz_ctx* ctx, hz_phase_time* out, int32_t cap, int32_t* count);

/* Continuous batching of point-source requests on one context (one mesh and
 * frequency; the factors stay resident). Multi-RHS processing is the paper's
 * motivation (Sec. "Introduction", Sec. "Conclusion"); the request loop
 * itself has no counterpart in the paper.
 * A server owns `slots` right-hand-side columns (<= max_block) and allocates
 * its blocks once, in hz_server_create. Requests (several sources each) are
 * queued by hz_server_submit; every hz_server_step admits queued sources
 * into free slots, runs one FGMRES restart cycle on all occupied slots
 * together, and retires the slots whose true residual reached rtol (or that
 * used maxit iterations). Each column has its own Krylov space and its
 * arithmetic does not depend on the other columns, so a request's
 * wavefields are the same alone and in any mix. The ids of finished
 * requests are written to done_ids, oldest first, at most cap per call (*ndone
 * of them); ids that do not fit are kept and returned by the next
 * hz_server_step calls, which return them even when no slot is active. Each
 * finished request is read once with hz_server_fetch (u [ns][n][2] host doubles; HZ_ENOTCONV if a column stopped
 * at maxit). Steps of servers of different contexts may be interleaved; a
 * server and its context are not thread-safe. Free a server (hz_server_free)
 * before its context (hz_free). Errors: HZ_EINVAL (bad
 * argument, unknown or unfinished request, duplicate id, source outside the
 * mesh), HZ_ENOMEM, HZ_ECUDA. */
typedef struct hz_server hz_server;
int hz_server_create(hz_ctx* ctx, int32_t slots, hz_server** out);
/* Device bytes one slot (right-hand-side column) of a server on ctx costs:
 * the server's blocks plus the context workspace of one column (Krylov basis,
 * preconditioner blocks, local sub-vectors of both levels). A caller admits by
 * device footprint by creating servers with budget / column_bytes slots. */
int hz_server_column_bytes(const hz_ctx* ctx, double* bytes);
int hz_server_submit(hz_server* srv, int64_t request_id, const double* src_xyz, const double* src_amp, int32_t ns);
int hz_server_step(hz_server* srv, int64_t* done_ids, int32_t cap, int32_t* ndone);
int hz_server_fetch(hz_server* srv, int64_t request_id, double* u, hz_stats* stats);
int hz_server_pending(const hz_server* srv, int32_t* queued, int32_t* active);
void hz_server_free(hz_server* srv);

/* Receiver sampling operator P of the FWI misfit: the value at x_k of the
 * P3 field u is sum_i w[k][i] u[idx[k][i]], with phi evaluated in the
 * lowest-index element containing x_k (the rule of the point-source load, so
 * P^T a is the load of point sources of amplitudes a at the receivers).
 *   rec_xyz [nr][3]; idx [nr][20] dofs (-1: Dirichlet dof or zero weight);
 *   w [nr][20]. Host only; HZ_EINVAL if a receiver lies outside the mesh. */
int hz_receiver_operator(const hz_ctx* ctx, const double* rec_xyz, int32_t nr, int32_t* idx, double* w);

/* Least-squares FWI misfit and its gradient with respect to the squared
 * slowness m_e = 1/c_e^2 of every element, by the adjoint-state method. The
 * paper's solver is the forward engine of frequency-domain FWI (Sec.
 * "Introduction"); it prints no gradient, the formula is the standard one:
 *   chi = 1/2 sum_s sum_k |(P u_s)_k - d_{s,k}|^2,  A u_s = F_s (point sources),
 *   A lambda_s = P^T conj(P u_s - d_s)   (A is complex symmetric),
 *   grad_e = -Re sum_s lambda_s^T (dA/dm_e) u_s,
 *   dA/dm_e = -omega^2 M_e - (i omega / (2 sqrt(m_e))) sum_{Robin faces f of e} B_f
 * on the element's non-Dirichlet dofs. Forward and adjoint solves use the
 * context's factors and options (2 ns solves).
 *   src_xyz [ns][3], src_amp [ns][2]: point sources as in hz_solve
 *   rec_xyz [nr][3]: receivers (hz_receiver_operator)
 *   d_obs   [ns][nr][2] observed data, host; NULL = zero data
 *   chi     misfit (may be NULL); grad [ne] host output
 *   d_syn   [ns][nr][2] host output P u_s (may be NULL)
 *   stats   iterations = max over all solves, ncols = 2 ns (may be NULL)
 * The first call uploads per-element data (dofs, volumes, Robin face areas,
 * m) that the context then keeps. Returns HZ_ENOTCONV if a solve stopped at
 * maxit (outputs computed from the last iterates). */
int hz_fwi_gradient(hz_ctx* ctx, const double* src_xyz, const double* src_amp, int32_t ns, const double* rec_xyz,
                    int32_t nr, const double* d_obs, double* chi, double* grad, double* d_syn, hz_stats* stats);

/* Host copy of A in CSR form: rowptr [n+1], col [nnz], val [nnz][2]. */
int hz_matrix_csr(const hz_ctx* ctx, int64_t* rowptr, int32_t* col, double* val);

/* Allocation-free Y = A X, for callers that cannot allocate device memory
 * when they call the library: code running where cudaMalloc/cudaFree are not
 * allowed (they synchronise the device), or processes whose device memory is
 * entirely managed by their own allocator. The paper has no counterpart; the
 * product is the one of hz_apply_A.
 *   X, Y   device pointers, [s][n][2] doubles (same layout as hz_apply_A)
 *   stream cudaStream_t the kernels are queued on (NULL: legacy default
 *          stream); the call returns without waiting for them
 * Its two [n][s] work blocks live in a file-scope device array of
 * 2 x HZ_NOALLOC_MAX_ENTRIES complex values (32 MiB). hz_setup, with the
 * context's device current, looks up the array's device address and keeps it
 * in the context; that lookup loads the array on the device (it then stays
 * there until the process exits), so the calls themselves allocate nothing.
 * The current device must be the one hz_setup ran on, else HZ_EINVAL.
 * n * s > HZ_NOALLOC_MAX_ENTRIES is refused with HZ_EINVAL before any launch;
 * HZ_ECUDA if hz_setup could not look the array up. All calls share the
 * array: calls whose kernels overlap on the GPU (other streams, other
 * threads, other contexts) race. Every call overwrites the entries it reads,
 * so no state carries over between calls. */
#define HZ_NOALLOC_MAX_ENTRIES 1048576
int hz_apply_A_noalloc(hz_ctx* ctx, const double* X, double* Y, int32_t s, void* stream);

void hz_free(hz_ctx* ctx);
const char* hz_strerror(int code);
const char* hz_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
