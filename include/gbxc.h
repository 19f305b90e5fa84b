/*
 * gbxc -- exchange-correlation integration on one GB300 (sm_103a).
 *
 * Computes E_xc, the potential matrix V_xc and the electron count N_el of a
 * spin-restricted density in a contracted Cartesian Gaussian basis by atomic
 * quadrature, following Williams-Young, de Jong, van Dam and Yang, "On the
 * Efficient Evaluation of the Exchange Correlation Potential on Graphics
 * Processing Unit Clusters" (Sec. 2.1-2.3, Algorithms 1-4).
 *
 * Conventions for every call:
 *   - Return value: GBXC_OK (0) or a negative GBXC_E* code; no call aborts or
 *     throws.  gbxc_last_error() gives a one-line message for the last failure
 *     on that context.
 *   - Units: bohr and hartree.
 *   - The caller owns every buffer it passes in or out; the library copies
 *     whatever it keeps.  Pointers marked "host or device" may point to host
 *     memory (pageable or pinned) or to device memory on the context's GPU;
 *     the library tells them apart with cudaPointerGetAttributes.
 *   - Matrices are N_b x N_b, row-major, float64.  Basis-function order is
 *     atom-major, then shell order as given to gbxc_load_basis, then the
 *     Cartesian components (l, m, n) of the shell with l descending, then m
 *     descending (xx, xy, xz, yy, yz, zz for L = 2).
 *   - A context is not thread-safe: calls on one context must be serialised by
 *     the caller.  Distinct contexts are independent.
 */
#ifndef GBXC_H
#define GBXC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBXC_OK 0
#define GBXC_EINVAL (-1)    /* bad argument (null pointer, size, index, enum) */
#define GBXC_ENOMEM (-2)    /* device or host allocation failed / footprint does not fit */
#define GBXC_ECUDA (-3)     /* a CUDA runtime call or a kernel launch failed */
#define GBXC_ETIMEOUT (-4)  /* a bounded wait expired */
#define GBXC_ENOTREADY (-5) /* the molecule has no grid yet, or a ticket is still running */
#define GBXC_ENOENT (-6)    /* unknown molecule id or ticket */

/* atomic partition function (Sec. 2.2) */
#define GBXC_BECKE 0
#define GBXC_SSF 1

/* exchange-correlation functional */
#define GBXC_SLATER 0       /* Slater (Dirac) exchange, LDA */
#define GBXC_PBE 1          /* PBE exchange + PBE correlation (PW92 inside), GGA */
#define GBXC_MVS_X 2        /* MVS exchange, a meta-GGA in rho, sigma and the kinetic energy
                               density tau = 1/2 sum P grad phi . grad phi (the meta-GGA
                               extension of Sec. 2.1); gbxc_integrate and
                               gbxc_integrate_batches, both precisions */
#define GBXC_PBE0_SL 3      /* the semi-local part of the PBE0 hybrid (Sec. 2.1 names hybrids):
                               3/4 PBE exchange + PBE correlation.  The remaining 1/4 exact
                               (Hartree-Fock) exchange is a four-centre integral, not a grid
                               quadrature, and is left to the caller; accepted wherever
                               GBXC_PBE is */

/* arithmetic of the integration */
#define GBXC_FP64 0         /* every step in float64 */
#define GBXC_MIXED 1        /* double-float (float32 pair) collocation and densities; both
                               contractions on the tensor cores as Ozaki-sliced bf16 products
                               (5 slices of 7 bits, 15 products, exact fp32 accumulator
                               levels); float64 weights, functional and accumulation */

/* kernel classes reported by gbxc_profile_read */
#define GBXC_K_WEIGHTS 0    /* partition weights (grid loading) */
#define GBXC_K_COLLOC 1     /* collocation Phi, grad Phi */
#define GBXC_K_XGEMM 2      /* X^j = P^j Phi^j (Eq. x_mat) */
#define GBXC_K_RHO_Z 3      /* rho, grad rho, functional, E/N, Z^j */
#define GBXC_K_VGEMM 4      /* V^j contraction and scatter into V_xc (Eqs. vxc_batch, vxc_inc) */
#define GBXC_K_FINISH 5     /* symmetrisation and fixed-order E/N reductions */
#define GBXC_K_PGATHER 6    /* P^j gather/split for the mixed form */
#define GBXC_K_OTHER 7       /* whole CUDA-graph launches of gbxc_integrate_many */
#define GBXC_K_SLICE 8       /* Ozaki slicing of the V-contraction operands (mixed form) */
#define GBXC_NKERNEL 9

#define GBXC_MAX_PRIM 8     /* primitives per shell */
#define GBXC_MAX_L 3        /* highest angular momentum (f) */

typedef struct gbxc_ctx gbxc_ctx;

#define GBXC_ANGULAR_PRODUCT 0  /* Gauss-Legendre in cos(theta) x trapezoid in phi */
#define GBXC_ANGULAR_LEBEDEV 1  /* Lebedev-Laikov rule (Sec. 2.2) */

/* Atomic quadrature and batching parameters (Sec. 2.2).
 *   nrad      Mura-Knowles radial points per atom
 *   ntheta    product rule: Gauss-Legendre nodes in cos(theta);
 *             Lebedev rule: its number of points, one of 6 14 26 38 50 86 110 146 170
 *             194 302 590 974 (degrees 3 ... 53; the paper's FG, UFG and SFG grids use
 *             302, 590 and 974)
 *   nphi      product rule: trapezoid nodes in phi (angular grid = ntheta * nphi points);
 *             ignored for a Lebedev rule
 *   partition GBXC_BECKE or GBXC_SSF
 *   max_batch batch threshold of the cuboid subdivision (the paper uses 512)
 *   eta       screening tolerance of Eq. rcut (the paper uses 1e-10)
 *   mk_alpha  Mura-Knowles radial scale (same for every element)
 *   angular   GBXC_ANGULAR_PRODUCT (0, the default of a zeroed struct) or
 *             GBXC_ANGULAR_LEBEDEV.  A Lebedev rule's points are its octahedral orbits
 *             expanded in a fixed order: orbits a1 (1,0,0), a2 (s,s,0), a3 (t,t,t),
 *             b (l,l,m), c (p,q,0), d (r,s,u), each kind by ascending generator; within
 *             an orbit the coordinate permutations in lexicographic order, for each the
 *             sign patterns +++, ++-, +-+, ..., ---, first occurrences only.          */
typedef struct {
    int nrad, ntheta, nphi;
    int partition;
    int max_batch;
    double eta;
    double mk_alpha;
    int angular;
} gbxc_grid_spec;

/* Sizes of a loaded molecule's plan. */
typedef struct {
    int natoms, nshell, nbf;
    long long npts;          /* total grid points N_g */
    int nbatch;              /* merged batches (Algorithm 3's final merge) */
    int nleaf;               /* batches before merging */
    long long nshell_entries;/* sum over batches of |S_j| in shells */
    long long nfunc_entries; /* sum over batches of N_b^j */
    long long ntiles;        /* 128-point tiles over all batches */
    double sum_mn2;          /* sum_j N_g^j (N_b^j)^2 */
    double work;             /* sum_j W_j of Eq. batch_work */
    double sum_mn;           /* sum_j N_g^j N_b^j (grid-point x function elements) */
    double sum_ms;           /* sum_j N_g^j |S_j| (grid-point x shell pairs of the collocation) */
    double sum_n2;           /* sum_j (N_b^j)^2 (elements of the gathered P^j) */
    int max_nfunc;           /* largest N_b^j */
} gbxc_plan_info;

/* Create a context on CUDA device `device` (device = -1 creates a host-only
 * context: basis and grid loading build the plan on the host and
 * gbxc_export_plan returns it, except the partition weights; no CUDA call is
 * made and integration returns GBXC_EINVAL).  `scratch_bytes` bounds the device
 * scratch used per integration (0 = half the free device memory at the first integration,
 * at most 128 GiB); work
 * that does not fit is processed in chunks of batches, like the paper's
 * device-memory-saturating subsets (Algorithm 2). */
int gbxc_create(gbxc_ctx **out, int device, size_t scratch_bytes);

/* Release every device and host resource of the context.  NULL is a no-op. */
void gbxc_destroy(gbxc_ctx *ctx);

/* Message of the last failure on `ctx` (never NULL; "" if none). */
const char *gbxc_last_error(const gbxc_ctx *ctx);

/* Register a molecule and its basis (Eq. gau_cart).
 *   xyz        natoms x 3 nuclear positions, bohr (host)
 *   Z          natoms nuclear charges (host; used for bookkeeping only)
 *   nshell     number of shells; for shell s:
 *   shell_atom[s]  atom index, shells must be grouped by atom in ascending atom order
 *   shell_L[s]     angular momentum 0..GBXC_MAX_L
 *   shell_nprim[s] primitives 1..GBXC_MAX_PRIM
 *   alpha, coeff   nshell x GBXC_MAX_PRIM exponents and contraction coefficients
 *                  (normalisation already folded into coeff; unused entries ignored)
 * On success *mol_out is the molecule id and *nbf_out the number of functions.
 * All inputs are host memory and are copied. */
int gbxc_load_basis(gbxc_ctx *ctx, int natoms, const double *xyz, const int *Z, int nshell,
                    const int *shell_atom, const int *shell_L, const int *shell_nprim,
                    const double *alpha, const double *coeff, int *mol_out, int *nbf_out);

/* The same with spherical shells (the paper's cc-pVDZ runs, Sec. 3): shell_pure[s] != 0 makes
 * a shell with L >= 2 carry the 2L+1 real solid harmonics S_Lm, m = -L..L, in Racah
 * normalisation (sqrt(4 pi/(2L+1)) r^L Y_Lm, the same norm as x^L), as combinations of its
 * Cartesian functions, e.g. for L = 2: sqrt3 xy, sqrt3 yz, z^2 - (x^2 + y^2)/2, sqrt3 xz,
 * sqrt3/2 (x^2 - y^2).  Functions are numbered shell by shell as before, a pure shell
 * contributing 2L+1.  shell_pure may be NULL (all Cartesian: gbxc_load_basis). */
int gbxc_load_basis_pure(gbxc_ctx *ctx, int natoms, const double *xyz, const int *Z, int nshell,
                         const int *shell_atom, const int *shell_L, const int *shell_nprim,
                         const int *shell_pure, const double *alpha, const double *coeff, int *mol_out,
                         int *nbf_out);

/* Build the molecular grid and the batch plan, and keep them on the device
 * (Sec. 2.2 and Algorithm 3; the paper reuses them across SCF iterations):
 * atomic grids, partition weights (computed on the GPU in float64), cuboid
 * batches, Algorithm 1 screening with Eq. rcut, the merge of equal shell
 * lists.  May be called again to replace the grid.  *npts_out and
 * *nbatch_out may be NULL. */
int gbxc_load_grid(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out,
                   int *nbatch_out);

/* The same as gbxc_load_grid with the grid expansion, the cuboid subdivision of every atom's
 * points and Algorithm 1 on every leaf run as device kernels (the batch merge and layout stay
 * on the host).  The resulting grid, batches and screening lists are identical, bit for bit,
 * to gbxc_load_grid's.  The paper plans on the host and points to moving Algorithm 3's batch
 * generation and screening to the GPU as the way to relieve its strong-scaling limit
 * (Algorithm 3 discussion; Conclusion).  GBXC_EINVAL for a host-only context or a grid of
 * 2^31 points or more. */
int gbxc_load_grid_device(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out,
                          int *nbatch_out);

/* Tracing and test hook: integrate batch `batch` alone (as gbxc_integrate_batches) and copy
 * its per-point intermediates out of the scratch slabs, point-major m x n row-major (m points
 * of the batch in batch order, n its functions in the batch's function order; both from
 * gbxc_export_plan / gbxc_plan_info_get): Phi and dPhi/dx, dPhi/dy, dPhi/dz as collocated
 * (Eq. gau_cart and its gradient), and Z (Eq. z_mat) as formed for the V contraction, in
 * float64 (double-float pairs summed for the mixed form).  Any output may be NULL.
 * functional GBXC_SLATER, GBXC_PBE or GBXC_PBE0_SL; GBXC_EINVAL if the batch needs more than one chunk. */
int gbxc_debug_batch(gbxc_ctx *ctx, int mol, int batch, const double *P, int functional, int precision,
                     double *phi, double *gx, double *gy, double *gz, double *z);

/* Plan files (checkpoint / resume of the resident grid): gbxc_save_plan writes the grid spec,
 * the points in batch order (x, y, z, w^q, parent atom, generation index) and the merged
 * batches with their shell lists of `mol` to `path`; gbxc_load_plan reads such a file for a
 * molecule with the same atoms and basis (checked by a hash) and makes it the molecule's
 * grid without re-planning (the partition weights are recomputed on the device; the
 * paper reuses grids and plans across SCF iterations, Sec. 2.2).  The file layout is the
 * host's native one.  GBXC_EINVAL for I/O errors, a foreign or corrupt file (every size,
 * pointer and index is validated before the molecule's grid is replaced), GBXC_ENOTREADY
 * for a molecule without a grid (save) or while requests are in flight (load). */
int gbxc_save_plan(gbxc_ctx *ctx, int mol, const char *path);
int gbxc_load_plan(gbxc_ctx *ctx, int mol, const char *path, long long *npts_out, int *nbatch_out);

/* Release everything the library holds for `mol` (basis, grid, partition weights, plan,
 * schedules and cached graphs that include it); the id is not reused.  The boundary's
 * counterpart of load_basis/load_grid (the resident per-molecule state of Sec. 2.3's
 * device memory management).  GBXC_ENOENT for an unknown id, GBXC_ENOTREADY while the
 * request server has requests queued or in flight. */
int gbxc_unload(gbxc_ctx *ctx, int mol);

/* Sizes of the plan of `mol` (after gbxc_load_grid). */
int gbxc_plan_info_get(gbxc_ctx *ctx, int mol, gbxc_plan_info *info);

/* Copy the plan to host buffers (any pointer may be NULL to skip it).
 * Point arrays are in the library's batch order (merged batch by merged
 * batch, points of a batch in the order the batching produced them):
 *   x, y, z, wq, w   npts float64: coordinates, unpartitioned weights w^q and
 *                    partitioned weights w = p_A w^q (Eq. num_int)
 *   parent           npts int32: atom whose quadrature holds the point
 *   point_index      npts int64: index of the point in the atom-major generation
 *                    order (atom, radial, theta, phi)
 *   batch_ptr        nbatch+1 int64 offsets into the point arrays
 *   shell_ptr        nbatch+1 int64 offsets into shell_idx
 *   shell_idx        nshell_entries int32 sorted shell lists S_j           */
int gbxc_export_plan(gbxc_ctx *ctx, int mol, double *x, double *y, double *z, double *wq,
                     double *w, int *parent, long long *point_index, long long *batch_ptr,
                     long long *shell_ptr, int *shell_idx);

/* Integrate E_xc, V_xc and N_el for density matrix P (Algorithm 4 over every
 * batch of the plan; Eqs. x_mat, eval_local_den, eval_local_den_grad,
 * eval_xc_batch, exc_batch, z_mat, vxc_batch, vxc_inc).
 *   P          nbf x nbf symmetric density matrix, host or device; read as given
 *   functional GBXC_SLATER, GBXC_PBE, GBXC_PBE0_SL, or GBXC_MVS_X (meta-GGA)
 *   precision  GBXC_FP64 or GBXC_MIXED (any batch size: batches with more than 1,184
 *              significant functions run the X contraction in exact K segments)
 *   Exc, Nel   host scalars (may be NULL)
 *   Vxc        nbf x nbf output, host or device (may be NULL); exactly symmetric
 *   stream     cudaStream_t to run on (NULL = the context's own stream); the call
 *              returns after the results are complete
 * GBXC_EINVAL when P holds a NaN or an infinity (checked on the device).      */
int gbxc_integrate(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision,
                   double *Exc, double *Vxc, double *Nel, void *stream);

/* Spin-unrestricted integration (the extension the paper notes for its method, Sec. 2.1):
 * spin densities rho_s = sum P^s_mu,nu phi_mu phi_nu from P^a and P^b, the spin-polarised
 * functional f(rho_a, rho_b, sigma_aa, sigma_ab, sigma_bb) (Slater exchange by spin scaling;
 * PBE exchange by spin scaling and PBE correlation with the PW92 spin interpolation), and
 * V^s = dE_xc/dP^s through Z^s = 1/2 w v_s Phi + w (2 s_ss grad rho_s + s_ab grad rho_s') .
 * grad Phi.  With P^a = P^b = P/2 the result equals gbxc_integrate's with P (V^a = V^b = V).
 *   Pa, Pb      nbf x nbf spin density matrices (host or device, symmetric)
 *   precision   GBXC_FP64, or GBXC_MIXED: the tensor-core form (both X contractions and both
 *               V contractions on the sliced bf16 operands; the densities and the
 *               spin-polarised functional in float64 from double-float sums)
 *   Exc, Nel    E_xc and the total electron count (may be NULL)
 *   Va, Vb      nbf x nbf outputs, host or device (may be NULL)
 *   stream      as gbxc_integrate */
int gbxc_integrate_uks(gbxc_ctx *ctx, int mol, const double *Pa, const double *Pb, int functional, int precision,
                       double *Exc, double *Va, double *Vb, double *Nel, void *stream);

/* As gbxc_integrate, restricted to merged batches [batch_begin, batch_end),
 * the device subset step of Algorithm 2.  E_batch and N_batch (host, may be
 * NULL) receive each batch's contribution, nbatch entries, zero outside the
 * range. */
int gbxc_integrate_batches(gbxc_ctx *ctx, int mol, const double *P, int functional,
                           int precision, int batch_begin, int batch_end, double *Exc,
                           double *Vxc, double *Nel, double *E_batch, double *N_batch,
                           void *stream);

/* Batching form: integrate several resident molecules in ONE CUDA graph launch.
 * Default (grouped) schedule: the molecules' plans are concatenated into one combined plan,
 * so each kernel launch (collocation, P^j slicing, the two contractions, rho/functional, Z)
 * covers the tiles of every molecule in a chunk of the device scratch, and a batch->molecule
 * map gives each batch its molecule's P, V accumulator and functional (the paper's
 * memory-saturating device subsets, Sec. 2.3, over all molecules at once).  The alternative
 * schedule (gbxc_set_schedule / gbxc_autotune with branches >= 1) spreads the molecules over
 * parallel graph branches by the greedy minimum-load rule of Algorithm 3 applied to the work
 * estimate of Eq. batch_work, each branch with its own stream and workspace.  The graph is
 * captured on the first call for a given (molecule list, precision, schedule) and replayed by
 * later calls with the same list (P and the functionals may change).  The workspaces of these
 * calls share one budget, fixed at the context's first such call: the scratch budget given to
 * gbxc_create, or else the default one capped by half the device memory then free after the part
 * of the single-call budget not yet allocated.  A NaN or
 * an infinity in any P returns GBXC_EINVAL.
 *   nmol          number of molecules (each id at most once)
 *   mol_ids[k]    molecule ids
 *   P[k]          nbf_k x nbf_k density matrices, host or device
 *   functional[k] GBXC_SLATER, GBXC_PBE or GBXC_PBE0_SL per molecule
 *   precision     GBXC_FP64 or GBXC_MIXED for all
 *   Exc, Nel      host arrays of nmol (may be NULL)
 *   Vxc[k]        outputs, host or device (Vxc or Vxc[k] may be NULL)
 * Returns after all results are complete. */
int gbxc_integrate_many(gbxc_ctx *ctx, int nmol, const int *mol_ids, const double *const *P,
                        const int *functional, int precision, double *Exc, double *const *Vxc,
                        double *Nel);

/* Autotuner of the batching form (no counterpart in the paper, which uses MAGMA's fixed
 * kernels): times gbxc_integrate_many on this molecule list for every candidate schedule --
 * the grouped launch (branches 0) and graph branch counts {1, 2, 4, 8, 16} (at most nmol),
 * and, for GBXC_MIXED, the tcgen05 GEMM N tile (128 functions with one TMEM accumulator set,
 * or 64 with two, which lets a tile's epilogue overlap the next tile's MMAs) -- by CUDA
 * events around the graph launch (best of
 * two replays after a capturing run), keeps the fastest for later gbxc_integrate_many calls
 * with the same (molecule list, precision) on this context, and returns it.
 *   arguments as gbxc_integrate_many (P is read; no results are returned)
 *   branches_out, tile_n_out  the chosen schedule (may be NULL)
 *   ms_out                    its device time per call in milliseconds (may be NULL)
 * Each candidate integrates the list three times, so a call costs about 3 x (number of
 * candidates) integrations. */
int gbxc_autotune(gbxc_ctx *ctx, int nmol, const int *mol_ids, const double *const *P,
                  const int *functional, int precision, int *branches_out, int *tile_n_out,
                  double *ms_out);

/* Sets the schedule gbxc_integrate_many uses for (molecule list, precision) on this context,
 * as gbxc_autotune would: `branches` 0 for the grouped launch, else that many graph branches
 * (1..64, at most nmol are used), and GEMM N tile `tile_n` (64 or 128; the float64 form
 * ignores it).  GBXC_EINVAL otherwise. */
int gbxc_set_schedule(gbxc_ctx *ctx, int nmol, const int *mol_ids, int precision, int branches, int tile_n);

/* Serving form: continuous batching of integration requests.
 * gbxc_serve_start allocates one device arena of `arena_bytes` (0 = the context's
 * scratch budget, or, when gbxc_create was given none, at most half the device memory free at
 * this call after the part of the single-call budget not yet allocated), creates `nslots`
 * streams and starts a scheduler thread.  Requests
 * (gbxc_submit) queue in arrival order; the scheduler admits the head of the queue as
 * soon as a slot is free and a contiguous region of the arena can hold the request's
 * device footprint (scratch of its batch schedule, P, V, partial sums and, for
 * GBXC_MIXED, the sliced P blocks), so requests that arrive while others run are admitted
 * as slots and memory free up and their work overlaps on the GPU.  Each request is
 * integrated exactly as gbxc_integrate would (same kernels), on its slot's stream.
 * gbxc_submit and gbxc_wait may be called from any thread while the server runs; other
 * calls on the context are serialised with the scheduler.  gbxc_load_grid is refused
 * (GBXC_ENOTREADY) while requests are queued or running.  gbxc_serve_stop finishes the
 * running requests, fails queued ones with GBXC_ENOTREADY and frees the arena. */
int gbxc_serve_start(gbxc_ctx *ctx, int nslots, size_t arena_bytes);
int gbxc_serve_stop(gbxc_ctx *ctx);

/* Queue one request; P (nbf x nbf, host) is copied before the call returns.
 * *ticket identifies the request for gbxc_wait. */
int gbxc_submit(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision, long long *ticket);

/* Wait up to timeout_s seconds for a request.  On completion fills Exc, Nel, Vxc (host,
 * nbf x nbf; any may be NULL) and *latency_s (submission to GPU completion, may be NULL),
 * forgets the ticket and returns the request's status; GBXC_ETIMEOUT if it is not done
 * yet (the ticket stays valid), GBXC_ENOENT for an unknown ticket. */
int gbxc_wait(gbxc_ctx *ctx, long long ticket, double timeout_s, double *Exc, double *Vxc, double *Nel,
              double *latency_s);

/* Queue length, requests on the GPU, requests completed since start, and the arena's free
 * and total bytes (any pointer may be NULL). */
int gbxc_serve_stats(gbxc_ctx *ctx, long long *queued, long long *running, long long *completed,
                     size_t *arena_free, size_t *arena_cap);

/* Float64 integration over every batch of `mol` for callers that cannot allocate
 * device memory (for example code running where cudaMalloc is unavailable or forbidden,
 * such as inside another library's memory pool or a pre-allocated real-time region).
 * This call itself allocates no device memory: its slab scratch is a static 64 MiB
 * device array inside the library (held by every GPU that loads the library until the
 * process exits), and everything else is caller-owned or was allocated when the
 * molecule was loaded.  The paper has no counterpart; it is a deployment variant of
 * gbxc_integrate with precision GBXC_FP64.
 *   P    nbf x nbf density matrix, DEVICE memory, read only
 *   Vxc  nbf x nbf DEVICE output; used as the accumulator, then symmetrised in place
 *   EN   2 doubles of DEVICE memory: {E_xc, N_el}
 *   stream  cudaStream_t (NULL = the context's stream)
 * P, Vxc and EN must be memory of the context's device (or managed memory); a buffer of
 * another device is refused with GBXC_EINVAL.
 * The work is queued on `stream` and the call returns without waiting: results are
 * ready when the stream reaches this point.  Because the call returns before the device
 * has looked at P, a NaN or an infinity in P cannot be reported by the return code; the
 * device checks P and then writes NaN to both E_xc and N_el, so such a result never looks
 * valid.  The first call on a device resolves the static array's device address
 * (cudaGetSymbolAddress) and caches it for the life of the process; make that first call
 * before any stream capture.  Calls share the one static array, and calls on the same
 * molecule also share its per-tile and per-batch E and N partial sums (allocated when the
 * grid was loaded), so calls whose work overlaps on the GPU (different streams, or
 * different contexts on one device) race and must not be issued concurrently.  A batch
 * whose tile needs more than 64 MiB of float64 slabs (more than about 10,900 padded
 * functions) is rejected with GBXC_ENOMEM. */
int gbxc_integrate_fp64_noalloc(gbxc_ctx *ctx, int mol, const double *P, int functional, double *Vxc,
                                double *EN, void *stream);

/* Measured arithmetic peaks of CUDA device `device`: float32 and float64 fused multiply-add
 * throughput in TFLOP/s (2 flops per FMA), from independent FMA chains on every SM timed with
 * CUDA events.  The paper has no counterpart: these are the denominators of the rooflines of
 * kernels bound by the plain ALUs (the double-float collocation runs on the float32 FMA pipe,
 * the float64 contractions on the float64 one).  Allocates and frees a small device buffer;
 * returns GBXC_EINVAL for NULL outputs, GBXC_ECUDA on a CUDA failure. */
int gbxc_measure_alu_peaks(int device, double *fp32_tflops, double *fp64_tflops);

/* Per-kernel-class accounting.  Launch counts are always kept; with
 * gbxc_profile_enable(ctx, 1) every kernel-class span is also bracketed by CUDA
 * events on the stream it runs on.  Enabling or disabling resets both.
 * gbxc_profile_read fills ms[GBXC_NKERNEL] (device milliseconds, NULL to skip)
 * and launches[GBXC_NKERNEL] (kernel launches, NULL to skip) since the last
 * reset; it synchronises with the recorded events. */
int gbxc_profile_enable(gbxc_ctx *ctx, int on);
int gbxc_profile_read(gbxc_ctx *ctx, double *ms, long long *launches);

#ifdef __cplusplus
}
#endif

#endif /* GBXC_H */
