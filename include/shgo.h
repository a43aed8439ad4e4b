/*
 * shgo.h - C ABI of the GB300 (sm_103a) library for nuclear-attraction integrals over
 * contracted solid-harmonic Gaussian orbitals (SHGOs), evaluated the way arXiv 2404.16245
 * describes: Gaussian product (Eq. 5), translation of both orbitals to the product centre P
 * by the solid-harmonic addition theorem (Eqs. 7-8, "vector uncoupling"), coupling of the two
 * harmonics at P (Clebsch-Gordan product rule, Supp. Eq. 4) and Boys functions (Eq. 12 and the
 * text after it), then contraction over primitives and nuclei (Eq. 11).
 *
 * Conventions shared by every entry point:
 *  - Lengths in bohr.  Orbitals follow Eq. 1 with Racah-normalised real solid harmonics
 *    (Eq. 2, Condon-Shortley phase): S_l0 = Y_l^0, S_{l,m>0} = (-1)^m sqrt2 Re Y_l^m,
 *    S_{l,-m} = (-1)^m sqrt2 Im Y_l^m, so S_11 = x, S_1,-1 = y, S_10 = z.
 *  - Coefficients multiply normalised primitives (N(l, alpha) of Eq. 1); each contracted
 *    function is renormalised to <phi|phi> = 1.
 *  - Function order: shells in input order, m = -l..l inside a shell.
 *  - V_ab = + sum_C Z_C <phi_a | 1/|r - C| | phi_b>  (no minus sign).
 *  - Device pointers are caller-owned CUDA device memory on the basis's device.  Calls that take
 *    a stream are asynchronous and stream-ordered (stream = a cudaStream_t, NULL = the legacy
 *    default stream).  Errors found before any launch are returned synchronously and the
 *    outputs are left untouched; a CUDA error is returned as SHGO_ERR_CUDA.
 *  - Failing calls leave a message for shgo_last_error() (thread-local).
 */
#ifndef SHGO_H
#define SHGO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SHGO_OK = 0,
  SHGO_ERR_INVALID_ARG = 1,   /* NULL pointer, negative count, non-finite or non-positive exponent */
  SHGO_ERR_UNSUPPORTED_L = 2, /* a shell with l > SHGO_LMAX */
  SHGO_ERR_OOM = 3,           /* device or host allocation failed */
  SHGO_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  SHGO_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
  SHGO_ERR_NUMERIC = 6        /* non-finite values detected */
} shgo_status;

#define SHGO_LMAX 8

typedef enum {
  SHGO_PREC_FP64 = 0,      /* every step in FP64 */
  SHGO_PREC_FP32_BULK = 1, /* nucleus loop (Eq. 11's per-nucleus factors and sums) in FP32 instructions:
                              every factor (pair-frame offset, T, the Boys Taylor step and recursions
                              from the FP64 grid, radial sums, unit-vector solid harmonics) an
                              unevaluated pair of FP32 numbers built with error-free transformations,
                              nucleus sums compensated (two-sum); block error ~1e-13 of the block's
                              largest element against FP64.  Gaunt coupling, primitive contraction,
                              translation and rotation in FP64 */
  SHGO_PREC_FP32_PLAIN = 2 /* the same kernel on single FP32 numbers (for error studies; ~1e-6) */
} shgo_precision;

/* Option flags (shgo_options.flags). */
#define SHGO_FLAG_BLOCK_SPARSE 1   /* V as the blocks of the shell pairs that have a primitive pair above the
                                      elementwise bound, packed (shgo_sparse_layout); single bases only */
#define SHGO_FLAG_NO_PRIM_BOUND 2  /* keep every primitive pair whose K_AB does not underflow: no
                                      elementwise bound (the method with no screening at all) */

typedef struct {
  int32_t precision; /* a shgo_precision value */
  int32_t device;    /* CUDA device ordinal, -1 = the current device */
  int32_t flags;     /* SHGO_FLAG_* bits, 0 = dense V with the primitive-pair bound */
} shgo_options;

/* Opaque basis: host copies of the shells, their normalised contraction coefficients, the
 * class-sorted shell-pair lists and the device buffers built from them.  Library-owned. */
typedef struct shgo_basis shgo_basis;

/* Nuclear positions: n rows of (x, y, z), device pointer, row-major, bohr. */
typedef struct {
  int64_t n;
  const double* xyz;
} shgo_centers;

/*
 * Build a basis of n_shells contracted shells (Eq. 1).
 *   l[s]          angular momentum of shell s, 0 <= l[s] <= SHGO_LMAX          (host)
 *   n_prim[s]     primitives of shell s, 1..64                                   (host)
 *   exponents     sum(n_prim) Gaussian exponents alpha > 0, shell after shell    (host)
 *   coefs         sum(n_prim) contraction coefficients of normalised primitives  (host)
 *   shell_xyz     n_shells x 3 centres a (bohr)                                  (host)
 *   opt           NULL = FP64 on the current device
 * The host arrays are copied; the caller keeps ownership.  On success *out receives a handle to
 * release with shgo_free().  Device memory for the pair lists, tables and the per-primitive-pair
 * coupling buffer is allocated here, on the selected device.
 */
shgo_status shgo_basis_create(int32_t n_shells, const int32_t* l, const int32_t* n_prim, const double* exponents,
                              const double* coefs, const double* shell_xyz, const shgo_options* opt,
                              shgo_basis** out);

/* One shard of a basis split over shard_count devices (one process or thread per device): the same basis,
 * keeping only the shell pairs of shard shard_index.  Inside each (la, lb) class the pairs, in the library's
 * pair order, are cut by their cumulative primitive-pair count (a pair's cost is its primitive-pair count
 * times the nuclei), so every shard gets about 1/shard_count of every class.  Calls on a shard compute only
 * its pairs: shgo_nuclear_attraction (and the overlap, two-centre Coulomb, derivative and field calls)
 * write only the shard's blocks of out, both triangles, and leave the other blocks untouched, so the shards'
 * outputs, each into a zeroed matrix, add up to the whole matrix (the blocks are disjoint: no collective,
 * the host gathers); the potential, its gradient and the contracted gradient return the shard's share of
 * the sum.  Four-centre integrals reject a shard (SHGO_ERR_INVALID_ARG).  shard_count = 1 is
 * shgo_basis_create.  Errors: those of shgo_basis_create; SHGO_ERR_INVALID_ARG for an index outside
 * 0..shard_count-1. */
shgo_status shgo_basis_create_shard(int32_t n_shells, const int32_t* l, const int32_t* n_prim,
                                    const double* exponents, const double* coefs, const double* shell_xyz,
                                    const shgo_options* opt, int32_t shard_index, int32_t shard_count,
                                    shgo_basis** out);

/* Primitive-pair bound.  With |S_lm(r)| <= |r|^l and the potential of a non-negative radial density peaking
 * at its centre, every element of one primitive pair's block is at most
 *   |c_i c_j| K_AB 4 pi int_0^inf (r + |PA|)^la (r + |PB|)^lb e^{-p r^2} r dr    per unit of total charge.
 * Primitive pairs whose bound is below 1e-20 are skipped by every kernel unless SHGO_FLAG_NO_PRIM_BOUND is
 * set, so an element of V moves by at most 1e-20 sum_C |Z_C| per skipped pair.
 *
 * Block-sparse output (SHGO_FLAG_BLOCK_SPARSE).  For bases whose dense nbf x nbf matrix is too large
 * (thousands of atoms): only the shell pairs with at least one primitive pair kept by the bound store a
 * block; every element of an omitted block is zero up to that bound.  Block q of the library's pair order
 * (shgo_pair_shells; a's l >= b's l, and a >= b within equal l) is (2 l_a + 1) x (2 l_b + 1) row-major at
 * out[offset[q]] with rows m_a = -l_a..l_a of shell a and columns m_b of shell b; offset[q] = -1 for an
 * omitted pair.  shgo_nuclear_attraction and shgo_nuclear_attraction_screened then write `out` in this
 * layout (ndoubles values, fully overwritten); the other integrals of such a basis stay dense.
 *   nblocks, ndoubles: host, may be NULL; offset: host array of shgo_basis_npairs values, may be NULL.
 * Errors: SHGO_ERR_INVALID_ARG (NULL basis, a basis without the flag). */
shgo_status shgo_sparse_layout(const shgo_basis* basis, int64_t* nblocks, int64_t* ndoubles, int64_t* offset);

/* Number of basis functions sum(2 l + 1) and of unique shell pairs n(n+1)/2. */
int64_t shgo_basis_nbf(const shgo_basis* basis);
int64_t shgo_basis_npairs(const shgo_basis* basis);

/*
 * V_ab = sum_C Z_C <phi_a|1/|r - C||phi_b> for every basis function pair (Eq. 11 with the one-
 * centre integral of Eq. 12 in its coupled form).
 *   centers   n nuclei, device [n][3] (n = 0 gives V = 0)
 *   charges   device [n], Z_C
 *   out       device [nbf][nbf] row-major FP64, fully overwritten (both triangles)
 *   stream    cudaStream_t the kernels are queued on
 * Asynchronous.  Not reentrant for one basis: calls on the same basis must be ordered (they
 * share the basis's coupling buffer).  A call with the same centers->xyz, charges and out pointers,
 * nucleus count and time limit as the basis's previous call replays that call's launches from a CUDA
 * graph (captured on an internal stream at the first repetition), which reads the arrays' current
 * contents; any other call launches directly and drops the graph.
 */
shgo_status shgo_nuclear_attraction(const shgo_basis* basis, const shgo_centers* centers, const double* charges,
                                    double* out, void* stream);

/* Same computation as shgo_nuclear_attraction, with CUDA events recorded on `stream` around
 * the two kernel phases; blocks until they complete and writes their device durations (ms):
 * phase_ms[0] = primitive-pair coupling blocks (Gaussian product, Boys, S_LM(C - P), nucleus
 * sums), phase_ms[1] = shell-pair blocks (Gaunt coupling, primitive contraction, translation,
 * write).  For measurement; the arithmetic and launches are those of the plain call. */
shgo_status shgo_nuclear_attraction_timed(const shgo_basis* basis, const shgo_centers* centers,
                                          const double* charges, double* out, void* stream, double* phase_ms);

/* Algorithmic FP64 operation counts (an FMA counts 2) of one shgo_nuclear_attraction call with
 * n_centers nuclei, per kernel phase as in shgo_nuclear_attraction_timed:
 *   flops[0]  per primitive-pair x nucleus: geometry, Boys (tabulated Taylor + recursion), the
 *             radial factors, S_LM(C - P) by recursion, and 2 per entry of R[L,M,k];
 *   flops[1]  per primitive pair: 2 per Gaunt term + 4 per W entry; per shell pair: building
 *             T_A, T_B and the two dense products T_A W T_B^T.
 * triples[0] receives the shell-triples (unique shell pairs x nuclei), triples[1] the primitive
 * triples (primitive pairs x nuclei). */
shgo_status shgo_basis_flops(const shgo_basis* basis, int64_t n_centers, double* flops, double* triples);

/* The same algorithmic FP64 model for shgo_nuclear_attraction_deriv (field = 0) or shgo_nuclear_field
 * (field = 1) of a single basis with n_centers nuclei: flops[0] the coupling kernel at la + lb + 1,
 * flops[1] the variant pair passes (raising, Gaunt coupling, translation, rotation) and the combine. */
shgo_status shgo_basis_deriv_flops(const shgo_basis* basis, int64_t n_centers, int32_t field, double* flops);

/* The same algorithmic FP64 model for shgo_esp (gradient = 0) or shgo_esp_gradient (gradient = 1) of a
 * single basis at n_points points: flops[0] the adjoint pass over the density (the pair kernel's count),
 * flops[1] the per-point pass (per live primitive pair and point: the point tables and the grouped sums).
 * SHGO_ERR_INVALID_ARG for a batch or a negative count. */
shgo_status shgo_basis_esp_flops(const shgo_basis* basis, int64_t n_points, int32_t gradient, double* flops);

/* Number of kernel launches one shgo_nuclear_attraction call on this basis makes (n > 0). */
int64_t shgo_basis_launches(const shgo_basis* basis);

/* Work queues and the time limit.  A call launches, per (la, lb) class, the coupling kernel (one block
 * per primitive pair at a time: Boys values, S_LM(C - P) and the nucleus sums) and then the pair kernel
 * (one block per shell pair at a time: Gaunt coupling, primitive contraction, translation, rotation,
 * write), the classes concurrently on a pool of streams.  Each launch is a grid of at most a few blocks
 * per SM whose blocks take their next primitive pair (shell pair) from a device work queue with one atomic
 * increment; in a batch the queue lists the work of molecules with more nuclei first.  No block waits on
 * another.
 *
 * Time limit of each launch, default none: before taking work a block compares the time since its
 * launch's first block started with the limit; once it has passed, the block takes no more work and the
 * call's device status becomes SHGO_ERR_TIMEOUT (the output is then incomplete).  seconds = 0 stops every
 * launch before any work (useful to exercise a caller's error path without a fault); INFINITY removes the
 * limit.  Applies to later shgo_nuclear_attraction, _batched and _screened calls on this basis or batch.
 * Errors: SHGO_ERR_INVALID_ARG (NULL basis, negative or NaN seconds). */
shgo_status shgo_basis_set_time_limit(shgo_basis* basis, double seconds);

/* Waits for the basis's last call that launched kernels and returns the device-side status of the calls
 * since the previous shgo_basis_sync: SHGO_OK, or SHGO_ERR_TIMEOUT when a launch of one of them reached the
 * time limit (shgo_basis_set_time_limit).  Reading the status clears it.  Errors: SHGO_ERR_INVALID_ARG
 * (NULL basis), SHGO_ERR_CUDA. */
shgo_status shgo_basis_sync(const shgo_basis* basis);

/* ---------------------------------------------------------------------------------------------
 * Allocation-free variant.  The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc, for example a process whose device memory belongs to an external pool
 * manager that forbids other allocations, or code that must never enter the CUDA allocator while
 * it runs.  shgo_basis_create allocates device memory, so such callers use this call instead.
 *
 * Same result as shgo_basis_create + shgo_nuclear_attraction + shgo_free, from the same host
 * basis arrays, device nuclei/charges and device output, on the current device.  It never calls
 * cudaMalloc, cudaFree or any allocating CUDA routine: the constant tables, this call's shells and
 * pair lists and its coupling buffer all live in one static device array of
 * SHGO_NOALLOC_SCRATCH_BYTES that the library holds on every GPU where it has been called, until the
 * process exits.  The CUDA driver loads the library's device code lazily (the default since CUDA
 * 12.2), so the array's memory is committed on a device when the first call runs there: make that
 * first call before an external pool manager takes the device's free memory.  If the device has no
 * room for the array at that point the call returns SHGO_ERR_OOM.  A problem whose shells, pairs and coupling buffer do not fit the part of that array left
 * after the tables (about 60 MiB; the 32-atom l <= 6 workload needs 24 MiB) is rejected with
 * SHGO_ERR_INVALID_ARG before any device work, and shgo_last_error() gives the sizes.
 *
 * The first call on a device does a one-time set-up (finds the array's device address with
 * cudaGetSymbolAddress and copies the tables into it, synchronously).  Later calls copy the shell
 * image from pageable host memory on
 * `stream`, which orders the copy after earlier work on that stream.  Every call reuses the same
 * array, which keeps the previous call's contents; nothing in it needs to start at zero.  Calls
 * whose device work overlaps (different streams or host threads on one device) race on the array.
 */
#define SHGO_NOALLOC_SCRATCH_BYTES (64ll * 1024 * 1024)
shgo_status shgo_nuclear_attraction_noalloc(int32_t n_shells, const int32_t* l, const int32_t* n_prim,
                                            const double* exponents, const double* coefs, const double* shell_xyz,
                                            const shgo_centers* centers, const double* charges, double* out,
                                            void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batches: many independent molecules in one call.  The shells of molecule m are the next
 * mol_nshells[m] shells of the arrays (same layout as shgo_basis_create); its nuclei are the next
 * mol_ncenters[m] rows of `centers`/`charges` at call time.  Pairs never cross molecules.  All
 * molecules' shell pairs of one (la, lb) class are computed by one launch per kernel, the classes
 * concurrently.  Release with shgo_free.
 * ------------------------------------------------------------------------------------------- */
shgo_status shgo_batch_create(int32_t n_mol, const int32_t* mol_nshells, const int64_t* mol_ncenters, int32_t n_shells,
                              const int32_t* l, const int32_t* n_prim, const double* exponents, const double* coefs,
                              const double* shell_xyz, const shgo_options* opt, shgo_basis** out);

/* Per molecule (host arrays of n_mol): its number of functions and the offset (in doubles) of its
 * row-major nbf_m x nbf_m block V_m in the batched output. */
shgo_status shgo_batch_layout(const shgo_basis* batch, int64_t* mol_nbf, int64_t* mol_out_offset);

/* Doubles of the batched output (sum of nbf_m^2), or -1 if `batch` is not a batch. */
int64_t shgo_batch_out_size(const shgo_basis* batch);

/* V_m for every molecule (Eq. 11 per molecule with its own nuclei).  centers [sum n_c][3] and
 * charges [sum n_c] are device arrays in molecule order; out is a device array of
 * shgo_batch_out_size doubles, fully overwritten.
 * The first call on a batch tunes, per (la, lb) class, the nucleus-chunk size of the coupling
 * kernel and the threads per block of the pair kernel by timing them on this work (it
 * synchronises `stream`; its output is exact).  The next call captures the whole launch sequence
 * into a CUDA graph on an internal stream; later calls with the same centers/charges/out pointers and
 * time limit replay it with one cudaGraphLaunch on `stream` (new pointers or a new limit re-capture).
 * Calls on one batch must be ordered, and batched calls on one device should come from one host thread
 * at a time. */
shgo_status shgo_nuclear_attraction_batched(shgo_basis* batch, const double* centers, const double* charges,
                                            double* out, void* stream);

/* Electrostatic potential of a density at arbitrary points (positive sign convention, as V):
 *   phi[k] = sum_{a,b} D_ab < phi_a | 1/|r - x_k| | phi_b >,
 * i.e. the attraction matrix of a unit point charge at x_k contracted with D (the electronic potential
 * of a one-particle density D is -phi).  Computed without forming any per-point matrix: the pair
 * kernel's linear map (Gaunt coupling of the one-centre integral, Eq. 12 corrected; translation,
 * Eqs. 7-8; rotation to the pair frame) is applied backwards to each density block once, and every
 * point then needs only the Boys values and solid harmonics of x_k - P per primitive pair (Eq. 11).
 * density: device, nbf x nbf row-major, symmetric (D_ab and D_ba both enter).  points: device
 * [n][3] (bohr).  phi: device [n], overwritten.  Single bases only (a batch, or a basis whose
 * coupling buffer is split into regions, gives SHGO_ERR_INVALID_ARG); uses the basis's coupling
 * buffer, so calls on one basis must be ordered with its other calls.  Asynchronous on `stream`. */
shgo_status shgo_esp(const shgo_basis* basis, const double* density, const shgo_centers* points, double* phi,
                     void* stream);

/* Gradient of that potential with respect to each point, grad[k][c] = d phi_k / d x_{k,c}
 *   = sum_{a,b} D_ab d/dx_{k,c} < phi_a | 1/|r - x_k| | phi_b >
 * (for a point charge q_k the force from the density's part of the energy sum_k q_k phi_k is -q_k grad[k];
 * for a nucleus, its Hellmann-Feynman term).  Same pipeline as shgo_esp with derivative tables per
 * point: gradients of the solid-harmonic polynomials (degree L -> L - 1, the raising/lowering of Eq. 3)
 * and dB_{L,k}/dT = -T^k/k! F_{L+k+1} (one more Boys order).  grad: device [n][3], overwritten.  Same
 * arguments, restrictions and errors as shgo_esp. */
shgo_status shgo_esp_gradient(const shgo_basis* basis, const double* density, const shgo_centers* points,
                              double* grad, void* stream);

/* Derivatives of V with respect to the basis-function centres:
 *   out[X][a][b] = d/dA_X sum_C Z_C < phi_a | 1/|r - C| | phi_b >,  X = x, y, z,
 * A the centre of phi_a's shell, the centre of phi_b's shell held fixed even where it coincides with A
 * (so out[X] is not symmetric; the derivative by the centre of phi_b is out[X][b][a]).  With the
 * nuclei's derivatives (shgo_nuclear_field) they sum to zero: out[X] + out[X]^T + field[X] = 0.
 * For phi_a = N S_la(r - A) exp(-alpha |r - A|^2) the derivative of the Gaussian product (Eq. 5) by A_X
 * has three parts: the lowered harmonic d_X S_la (a combination of S_{la-1,M}, Eq. 3's lowering), the
 * factor -2 mu (A - B)_X (mu = alpha beta / p) of K_AB, and 2 alpha (r - P)_X times the product, which
 * raises the one-centre integral of Eq. 12 to order la + lb + 1 (Eq. 3's product of S_1 with S_L).  Each
 * part runs through the steps of V (coupling at la + lb + 1, Gaunt coupling, translation, rotation) in
 * FP64, whatever the basis's precision.
 * centers, charges: device, as for shgo_nuclear_attraction.  out: device, 3 x nbf x nbf doubles
 * (component-major, each nbf x nbf row-major), fully overwritten.  Single bases only (a batch gives
 * SHGO_ERR_INVALID_ARG).  Allocates its work arrays stream-ordered on `stream` (about
 * n_r(la + lb + 1) doubles per primitive pair and 9 blocks per shell pair; SHGO_ERR_OOM when they do not
 * fit).  The time limit of shgo_basis_set_time_limit does not apply.  Asynchronous on `stream`; calls on
 * one basis must be ordered with its other calls.  Errors: SHGO_ERR_INVALID_ARG, SHGO_ERR_OOM,
 * SHGO_ERR_CUDA. */
shgo_status shgo_nuclear_attraction_deriv(const shgo_basis* basis, const shgo_centers* centers,
                                          const double* charges, double* out, void* stream);

/* Gradient of E = sum_{a,b} P_ab V_ab with respect to the centre of every shell (the nuclear-attraction part of
 * the basis-function force), without forming the derivative matrices:
 *   grad[s][X] = sum_{a in s} sum_b (P_ab + P_ba) dV_ab/dA_X,   A the centre of shell s,
 * i.e. dE/dA_X when only shell s moves; the shells on one atom add up to that atom's basis-function term.  The
 * nuclei's own term is dE/dC_X = Z_C times shgo_esp_gradient at C for the same (symmetric) density, and
 * translational invariance gives sum_s grad[s] + sum_C dE/dC = 0.  The same pipeline as
 * shgo_nuclear_attraction_deriv; each shell pair's elements are weighted by P and summed on the device (one
 * warp per pair, a fixed order), then each shell adds its pairs in pair order: the result does not depend on
 * the schedule.  density: device, nbf x nbf row-major (any matrix).  grad: device [n_shells][3], overwritten.
 * Same arguments, restrictions and errors as shgo_nuclear_attraction_deriv (no nbf^2 output is allocated). */
shgo_status shgo_nuclear_attraction_gradient(const shgo_basis* basis, const double* density,
                                             const shgo_centers* centers, const double* charges, double* grad,
                                             void* stream);

/* Field integrals of the nuclei (derivative of V by the nucleus positions, summed):
 *   out[X][a][b] = sum_C Z_C d/dC_X < phi_a | 1/|r - C| | phi_b >   (symmetric in a, b).
 * The matrix of one nucleus C (the Hellmann-Feynman force integrals) is the call with that nucleus alone
 * and Z_C = 1.  The one-centre integral of Eq. 12 depends on C - P only, and its derivative is the
 * integral of the differentiated integrand d_X [r^{2k} S_LM(r) e^{-p r^2}], which the l +- 1 steps of Eq. 3
 * write as one-centre integrals of order la + lb + 1; the rest is the pipeline of V.  Same arguments,
 * layout, restrictions and errors as shgo_nuclear_attraction_deriv (3 blocks per shell pair). */
shgo_status shgo_nuclear_field(const shgo_basis* basis, const shgo_centers* centers, const double* charges,
                               double* out, void* stream);

/* Overlap matrix S_ab = <a|b> of a basis or of every molecule of a batch (Eqs. 9-10): both
 * Gaussians of a pair translated to the product centre P (Eq. 7), where the one-centre integral is
 * diagonal in (l, m) by the orthogonality of Eq. 10, then rotated from the pair frame back to the
 * molecular frame.  out: device array, row-major nbf x nbf for a basis (symmetric, fully
 * overwritten), the batched layout of shgo_batch_layout for a batch.  Asynchronous on `stream`;
 * no nuclei are involved.  Errors: SHGO_ERR_INVALID_ARG (NULL basis or out), SHGO_ERR_CUDA. */
shgo_status shgo_overlap(const shgo_basis* basis, double* out, void* stream);

/* Two-centre Coulomb integrals (a|b) = int int phi_a(r1) phi_b(r2) / |r1 - r2| (the two-centre case of the
 * electron-repulsion integrals, Eqs. 13-15; the Coulomb metric of density fitting) of a basis or of every
 * molecule of a batch.  With Eq. 3 each orbital is a solid-harmonic derivative of an s Gaussian with
 * respect to its centre, so (a|b) is S_la(grad_R) S_lb(grad_R) applied to the s-s integral, a function of
 * |A - B|^2 through F_0; the product rule of solid harmonics (the Gaunt coupling) and Hobson's theorem
 * turn it into sum_{L,M} G 2^L S_LM(A - B) times Boys values F_{L+k+j}.  Computed in FP64 whatever the
 * basis's precision option.  out: as for shgo_overlap (symmetric, fully overwritten).  Asynchronous on
 * `stream`.  Errors: SHGO_ERR_INVALID_ARG (NULL basis or out), SHGO_ERR_CUDA. */
shgo_status shgo_coulomb_2c(const shgo_basis* basis, double* out, void* stream);

/* Four-centre electron-repulsion integrals (ab|cd) = int int phi_a(r1) phi_b(r1) phi_c(r2) phi_d(r2) /
 * |r1 - r2| (Eqs. 13-15) of a single basis (not a batch) whose shells all have l <= 4.  Each pair is
 * translated to its product centre (Eq. 7) and its harmonics coupled there (Gaunt coefficients); the
 * r^{2k} factors of the coupled terms become powers of the Laplacian, so with Eq. 3 both pairs are
 * harmonic differential operators applied to the s-s integral of the two product Gaussians, which the
 * product rule and Hobson's theorem evaluate as sum_{L,M} G 2^L S_LM(P - Q) times Boys values F_N(rho
 * |P - Q|^2), rho = pq/(p + q).  FP64 whatever the basis's precision option.  out: device array of
 * nbf^4 doubles, row-major, out[((i nbf + j) nbf + k) nbf + l] = (ij|kl), fully overwritten (every
 * unique quartet once, written to its eight permutations).  A per-call device buffer of
 * sum over primitive pairs of (2la+1)(2lb+1) C(la+lb+3, 3) doubles, plus a scratch region of partial
 * blocks per pool stream (at most 8M doubles each, or the count in the environment variable
 * SHGO_ERI_SCRATCH_DOUBLES; larger work is cut into pieces that fit), is taken from the device's default
 * stream-ordered pool and returned on `stream`.  Asynchronous on `stream`.  Errors: SHGO_ERR_INVALID_ARG
 * (NULL basis or out, a batch, nbf > 40000), SHGO_ERR_UNSUPPORTED_L (a shell with l > 4), SHGO_ERR_OOM,
 * SHGO_ERR_CUDA. */
shgo_status shgo_eri(const shgo_basis* basis, double* out, void* stream);

/* Coulomb and exchange matrices of a density from the same integrals, without storing them:
 * J[p][q] = sum_rs (pq|rs) D[r][s] and K[p][r] = sum_qs (pq|rs) D[q][s], all indices over the basis
 * functions (Eqs. 13-15 as in shgo_eri; basis with l <= 4, not a batch).  density: device nbf x nbf
 * row-major (any matrix; symmetric for the usual closed-shell use).  J, K: device nbf x nbf row-major,
 * fully overwritten; either may be NULL, not both.  Each unique integral is formed once and added to
 * the entries of its distinct permutations with atomic additions, so the last bits of J and K may vary
 * from call to call.  Scratch as for shgo_eri; no nbf^4 storage.  Asynchronous on `stream`.
 * Errors: SHGO_ERR_INVALID_ARG (NULL basis, density or both outputs, a batch), SHGO_ERR_UNSUPPORTED_L,
 * SHGO_ERR_OOM, SHGO_ERR_CUDA. */
shgo_status shgo_eri_jk(const shgo_basis* basis, const double* density, double* J, double* K, void* stream);

/* Per (la, lb) class (measurement): number of classes of a basis (-1 for NULL); for class c
 * (0 <= c < nclasses, in the library's launch order) its la >= lb in la_lb[2] and, for n_centers
 * nuclei, stats[4] = shell-triples, integrals (shell-triples x (2la+1)(2lb+1)), algorithmic flops of
 * the coupling kernel and of the pair kernel (FMA = 2 flops).  Errors: SHGO_ERR_INVALID_ARG. */
int32_t shgo_basis_nclasses(const shgo_basis* basis);
shgo_status shgo_basis_class_stats(const shgo_basis* basis, int64_t n_centers, int32_t c, int32_t* la_lb,
                                   double* stats);

/* V as shgo_nuclear_attraction (or, for a batch, shgo_nuclear_attraction_batched with centers->n =
 * all its nuclei) computes it, but with the classes run one after another on `stream` and the
 * device time of each class's coupling and pair kernels written to ms[2 c], ms[2 c + 1] (host array
 * of 2 x nclasses).  Blocks until done.  Bases whose coupling buffer is split into regions are
 * rejected (SHGO_ERR_INVALID_ARG). */
shgo_status shgo_nuclear_attraction_class_timed(const shgo_basis* basis, const shgo_centers* centers,
                                                const double* charges, double* out, void* stream, double* ms);

/* Measurement: the fused multiply-add rate of the current GPU's FP64 pipe (precision = SHGO_PREC_FP64) or
 * FP32 pipe (SHGO_PREC_FP32_BULK or SHGO_PREC_FP32_PLAIN), the denominator of the library's roofline
 * fractions (the paper states no hardware rate).  A grid of 2048 threads per SM, each running eight
 * independent multiply-add chains of 4 x iters steps, is launched once to warm up (iters / 16 + 1) and once
 * timed with CUDA events on `stream`; blocks until done.  flops_per_s receives 2 x FMAs per second of the
 * timed launch and ms its duration.  Takes a small scratch array from the device's default stream-ordered
 * pool.  Errors: SHGO_ERR_INVALID_ARG (NULL output, iters outside 1..2^32, unknown precision),
 * SHGO_ERR_OOM, SHGO_ERR_CUDA. */
shgo_status shgo_measure_fma_rate(int32_t precision, int64_t iters, void* stream, double* flops_per_s, double* ms);

/* The same measurement with a chosen launch shape: `chains` independent chains per thread (4, 8 or 16) and
 * threads_per_sm threads on every SM (a multiple of 256, at most 2048); shgo_measure_fma_rate is chains = 8,
 * threads_per_sm = 2048.  A sweep over shapes shows whether the rate is the pipe's or the launch's.
 * Errors as shgo_measure_fma_rate, plus SHGO_ERR_INVALID_ARG for a shape outside those values. */
shgo_status shgo_measure_fma_rate_shape(int32_t precision, int64_t iters, int32_t chains, int32_t threads_per_sm,
                                        void* stream, double* flops_per_s, double* ms);

/* Release a basis and its device memory (synchronises its device).  NULL-safe. */
void shgo_free(shgo_basis* basis);

/* Message of the last failing call on this thread ("" if none). */
const char* shgo_last_error(void);

/* ---------------------------------------------------------------------------------------------
 * Host-side views of the library's own tables and scalar algorithms, for testing them against
 * the mathematics without a GPU.  None of these is used on the device path.
 * ------------------------------------------------------------------------------------------- */

/* Real solid harmonics S_lm(r), m = -l..l, of Eq. 2 by the library's recursion:
 * out[p * (2l+1) + m + l] for the npts points xyz[3p..3p+2].  l <= 2 * SHGO_LMAX + 1. */
shgo_status shgo_host_solid_harmonics(int32_t l, int64_t npts, const double* xyz, double* out);

/* Real coupling coefficient G with S_{l1 m1}(r) S_{l2 m2}(r) = sum_{L,M} G r^{l1+l2-L} S_{LM}(r)
 * (the Clebsch-Gordan product rule behind Supp. Eq. 4, mapped to real harmonics).  l1, l2 <= 8. */
double shgo_host_gaunt(int32_t l1, int32_t m1, int32_t l2, int32_t m2, int32_t L, int32_t M);

/* Real translation coefficient E with S_{la,ma}(x + y) = sum E S_{l1,m1}(x) S_{la-l1,nu}(y):
 * the addition theorem of Eq. 7 with the vector-coupling coefficients of Eq. 8, mapped to real
 * harmonics.  la <= 8. */
double shgo_host_translation(int32_t la, int32_t ma, int32_t l1, int32_t m1, int32_t nu);

/* F_n(T), n = 0..nmax (nmax <= 2 * SHGO_LMAX + 1), by the device algorithm (tabulated Taylor
 * expansion and downward recursion below T = 40, asymptotic start and upward recursion above). */
shgo_status shgo_host_boys(int32_t nmax, double T, double* F);

/* The derivative integrals' steps on one coupling block, from the device tables.  r1 holds one-centre
 * integrals R'[L, M, k] of order lam + 1 (n_r(lam + 1) = (lam+2)(lam+3)(lam+4)/6 entries, ordered by L, then
 * M = -L..L, then k = 0..(lam + 1 - L)/2); raised and field receive n_r(lam) entries of order lam:
 *   raised[L, M, k] = the integral with r^{2k} S_LM(r) replaced by x_c r^{2k} S_LM(r),
 *   field[L, M, k]  = the integral with r^{2k} S_LM(r) e^{-p r^2} replaced by its derivative d/dx_c,
 * c = comp (0, 1, 2 = x, y, z).  lam <= 2 * SHGO_LMAX. */
shgo_status shgo_host_deriv_transform(int32_t lam, int32_t comp, double p, const double* r1, double* raised,
                                      double* field);

/* The shard of every shell pair of a single basis split over shard_count shards (shgo_basis_create_shard),
 * in the library's pair order (shgo_pair_shells), on the host.  *npairs: in, the room in shard; out, the
 * number of pairs (shard is written only when the room suffices; shard may be NULL to ask for the count). */
shgo_status shgo_host_shard_of_pairs(int32_t n_shells, const int32_t* l, const int32_t* n_prim, int32_t shard_count,
                                     int64_t* npairs, int32_t* shard);

/* Lowering coefficients: d/dx_c S_lm(r) = sum_M' w[M' + l - 1] S_{l-1,M'}(r), 1 <= l <= SHGO_LMAX;
 * w receives 2l - 1 values. */
shgo_status shgo_host_deriv_lowering(int32_t l, int32_t comp, int32_t m, double* w);

/* Coefficient a_{k,j}(L) of the k-fold Laplacian of a solid harmonic times a radial function:
 * Laplacian^k [S_LM(R) f(u)] = S_LM(R) sum_j a_{k,j}(L) u^j f^{(k+j)}(u), u = |R|^2, as the two- and
 * four-centre Coulomb kernels use it (L <= 2 SHGO_LMAX, j <= k <= SHGO_LMAX; 0 outside). */
double shgo_host_laplacian_coef(int32_t L, int32_t k, int32_t j);

/* Coefficient eps_{k,n}(L) of r^{2k} S_LM(r) e^{-p r^2} = sum_n eps_{k,n}(L) p^{-(k+n)} Laplacian^n
 * [S_LM(r) e^{-p r^2}] (the four-centre kernels; L <= 2 SHGO_LMAX, n <= k <= SHGO_LMAX; 0 outside). */
double shgo_host_eri_eps(int32_t L, int32_t k, int32_t n);

#ifdef __cplusplus
}
#endif
#endif /* SHGO_H */
