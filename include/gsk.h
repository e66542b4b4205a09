/*
 * gsk.h -- C ABI of libgsk, a GB300 (sm_103a) solver for the generalized
 * shifted linear equations of Hoshi et al., "Extremely scalable algorithm
 * for 10^8-atom quantum material simulation on the full system of the K
 * computer" (SC16, arXiv:1609.08377).
 *
 * For every requested basis column j the library solves
 *     (z_k B - A) x = e_j            for all shifts z_k          (Eq. EQ-SHIFT-EQ-J)
 * with one Krylov subspace shared by all shifts (Sec. III-B), where A (the
 * Hamiltonian) is real symmetric and B (the overlap) is symmetric positive
 * definite (Sec. II-A, Eq. EQ-GEV-EQ). It returns the Green's-function
 * elements G_ij(z_k) = [(z_k B - A)^{-1}]_ij (Eq. EQ-EIG-X=GB) for the rows
 * i of A's pattern in column j (nearsightedness, Sec. II-B), and from them the
 * density-matrix elements rho_ij by quadrature of Eq. EQ-DM-GREEN-FN with the
 * Fermi function of Eq. EQ-FD-FUNC.
 *
 * Conventions for every entry point:
 *  - Return value: GSK_OK (0) or a negative GSK_E* code. No call traps,
 *    aborts or exits; after an error the handle stays usable unless the error
 *    is GSK_ECUDA with a sticky CUDA error.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the device that was current at gsk_create.
 *  - Complex numbers are stored as interleaved pairs of doubles (re, im).
 *  - Indices are 0-based and refer to the caller's original ordering.
 *  - Calls on one handle are not thread safe; different handles are
 *    independent.
 *
 * Bounds-checked build: libgsk compiled with -DGSK_DEBUG (build.py's
 * debug build, libgsk_debug.so) has the same entry points. Its solve kernels
 * test every block-layout, tile and work-queue index before they use it; a
 * failed test records the first offence and skips the access (or sends it to
 * a valid row), so no kernel faults or traps on a bad index. gsk_solve and
 * gsk_spmm then return GSK_EBOUNDS and gsk_stats.debug_code / debug_index
 * name the check and the index (results are then unspecified); gsk_spmm
 * waits for its kernels in that build. The check codes:
 *    1  atom index, orbital count or own rows of an atom (gather products)
 *    2  neighbour-entry range or value range of an atom (gather products)
 *    3  neighbour row outside the rows of X (gather products)
 *   10  tile header: a copy outside the tile arrays, the values or the stage
 *       buffers, or a misaligned bulk copy (staged product, producers)
 *   11  row-run piece outside X or the stage's row buffer (producers)
 *   12  a warp's atom list outside the tile's descriptors (consumers)
 *   13  atom descriptor: own rows, values or neighbour indices outside the
 *       stage (consumers)
 *   14  shared row of a neighbour outside the stage's row buffer (consumers)
 *   20  work-queue entry that is not a job index
 *   21  a lane's job index outside the solve's columns
 *   22  row of e_j outside [0, M)
 *   23  pattern size of a column above the per-lane buffers
 *   24  pattern row outside [0, M) (shift recurrences)
 * The normal build compiles every check away.
 */
#ifndef GSK_H
#define GSK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----- call-level status codes ----------------------------------------- */
#define GSK_OK 0
#define GSK_EINVAL (-1)     /* bad shape, index, pointer, option or non-finite value */
#define GSK_ENOTSPD (-2)    /* B fails the positive-diagonal / diagonal-dominance check */
#define GSK_ENOMEM (-3)     /* device or host allocation failed */
#define GSK_ECUDA (-4)      /* a CUDA runtime call failed */
#define GSK_ETIMEOUT (-5)   /* a bounded device wait gave up */
#define GSK_ENOTSUP (-6)    /* option combination not supported (e.g. FP64 with 128 lanes) */
#define GSK_EBOUNDS (-7)    /* bounds-checked build only: an index check failed (see gsk_stats) */

/* ----- per-column status codes (status[] of gsk_solve) -------------------- */
#define GSK_CONVERGED 0      /* every shift reached the residual tolerance */
#define GSK_NOT_CONVERGED 1  /* max_iter reached; G holds the last iterate */
#define GSK_BREAKDOWN 2      /* beta^2 <= 0 or a non-finite scalar (e.g. B not SPD) */
#define GSK_TIMEOUT 3        /* the column was not finished within the step cap */

/* ----- option values ------------------------------------------------------ */
#define GSK_FP64 0           /* every product and vector update in FP64 */
#define GSK_MIXED 1          /* FP32 inner B-solve, FP64 residual refinement, FP64 Lanczos */
#define GSK_MIXED_DF 2       /* as GSK_MIXED, with the FP64-accuracy parts (A-products, refinement
                                residuals, Lanczos vectors, inner products) in double-float
                                arithmetic: pairs of FP32 numbers, 48-bit significand */

#define GSK_SPMM_AUTO 0      /* inner-CG products: the autotuner's pick, else staged at 32 lanes (default) */
#define GSK_SPMM_GATHER 1    /* every product by the per-atom gather kernel */
#define GSK_SPMM_STAGED 2    /* FP32 inner-CG products: tile rows staged in shared memory (mixed modes) */

#define GSK_SCHED_FIFO 0     /* columns enter the work queue in the given order */
#define GSK_SCHED_LEARNED 1  /* longest predicted iteration count first (needs a model) */

typedef struct gsk_ctx* gsk_handle;

/* Sparse symmetric matrix in CSR form (host memory, caller-owned, read only
 * during gsk_create). row_ptr has n_rows+1 entries, col_idx/val row_ptr[n]
 * entries; column indices within a row must be ascending and unique. */
typedef struct {
  int32_t n_rows;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
} gsk_csr;

/* Orbital-block map (Sec. II-C: basis index i <-> (atom I, orbital alpha)).
 * Atom I owns rows orb_offset[I] .. orb_offset[I] + orb_count[I] - 1; the
 * offsets must tile 0..n_rows-1 in increasing order; orb_count is 1 or 4.
 * pos (optional, may be NULL) holds 3*n_atoms coordinates used only to order
 * atoms along a space-filling curve for memory locality. Host memory, read
 * only during gsk_create. */
typedef struct {
  int32_t n_atoms;
  const int32_t* orb_offset;
  const int8_t* orb_count;
  const double* pos;
} gsk_orbmap;

/* Solver options. Zero-initialise and set what you need; gsk_default_options
 * fills the defaults listed here. */
typedef struct {
  int32_t precision;    /* GSK_FP64 (default), GSK_MIXED or GSK_MIXED_DF */
  double tol;           /* relative residual ||e_j - (z B - A) x||_2 for every shift; default 1e-8 */
  int32_t max_iter;     /* Lanczos steps per column; default 20000 */
  int32_t batch_w;      /* lanes (columns in flight): 32, 64 or 128; 0 = autotune (default) */
  int32_t refine;       /* mixed modes only: 1 = FP64-accurate residual correction of each B-solve (default), 0 = none */
  int32_t sched;        /* GSK_SCHED_FIFO (default) or GSK_SCHED_LEARNED (model set with gsk_set_sched_model) */
  double inner_tol;     /* relative residual of each B-solve; 0 = default (1e-12 FP64, 3e-6 per FP32 pass) */
  int32_t max_inner;    /* CG iteration cap per B-solve pass; default 200 */
  int32_t use_graph;    /* 1 = run the solve as one captured CUDA graph with device-side loops (default) */
  void* stream;         /* cudaStream_t to run on; NULL = the legacy default stream */
  int32_t spmm_kernel;  /* GSK_SPMM_AUTO (default), GSK_SPMM_GATHER or GSK_SPMM_STAGED: how the
                           FP32 products with B of the mixed modes' inner CG run. The gather
                           kernel reads every neighbour row per atom through the caches; the
                           staged kernel cuts the atoms (space-filling-curve order) into tiles
                           whose neighbour rows fit in shared memory and copies each tile's
                           rows, values and indices there once, asynchronously, two tiles in
                           flight. Both give the same product up to FP32 rounding order;
                           GSK_SPMM_STAGED on a non-mixed solve returns GSK_ENOTSUP. */
} gsk_options;

/* Fill *opt with the defaults above. */
void gsk_default_options(gsk_options* opt);

/* Build a solver handle from A, B (same pattern, symmetric) and the orbital
 * map. Copies the matrices to the device in the library's block layout
 * (FP64, plus FP32 and FP32-pair copies for the mixed modes). Returns GSK_EINVAL for malformed
 * input or non-finite values, GSK_ENOTSPD when some B_ii <= 0 or a row of B is
 * not strictly diagonally dominant (a sufficient test for positive
 * definiteness; the library requires it). The handle owns every device
 * buffer; *out is NULL on failure. The current CUDA device is bound to the
 * handle. */
int gsk_create(const gsk_csr* A, const gsk_csr* B, const gsk_orbmap* map, gsk_handle* out);

/* Release the handle and all its device memory. Accepts NULL. */
int gsk_destroy(gsk_handle h);

/* Matrix dimension M and number of stored entries of A. */
int gsk_dims(gsk_handle h, int32_t* M, int64_t* nnz);

/* offsets[c] = sum_{c' < c} |P(cols[c'])| for c = 0..n_cols, where P(j) is the
 * pattern of column j of A (host arrays). This is the layout of G and rho:
 * element (i, c, k) with i the t-th entry of CSR row cols[c] of A lives at
 * (offsets[c] + t) * n_shifts + k. */
int gsk_pattern_offsets(gsk_handle h, int32_t n_cols, const int32_t* cols, int64_t* offsets);

/* Solve (z_k B - A) x = e_j for j in cols and every shift, with the shifted
 * B-inner-product Lanczos method (one Krylov subspace per column shared by
 * all shifts, Sec. III-B), and write G_ij(z_k) for i in P(j).
 *
 *   n_shifts  S >= 1
 *   z         host, 2*S doubles: shifts (re, im); Im z_k > 0 required unless
 *             eta is given
 *   eta       host, n_cols doubles or NULL: if given, column c uses the
 *             shifts Re z_k + i*eta[c] (eta[c] > 0)
 *   cols      host, n_cols distinct column indices in [0, M)
 *   G         device (or host) buffer of offsets[n_cols]*S complex doubles
 *             (see gsk_pattern_offsets); host buffers are staged through
 *             device memory
 *   iters     host, n_cols: Lanczos steps taken per column (may be NULL)
 *   status    host, n_cols: GSK_CONVERGED ... per column (may be NULL)
 *   resid     host, n_cols: max over shifts of the residual estimate (may be NULL)
 *
 * The call is synchronous: it returns after the results are written.
 * Returns GSK_EINVAL for bad arguments (nothing is written). */
int gsk_solve(gsk_handle h, int32_t n_shifts, const double* z, const double* eta,
              int32_t n_cols, const int32_t* cols, const gsk_options* opt,
              double* G, int32_t* iters, int32_t* status, double* resid);

/* rho_ij = -(1/pi) * sum_k w_k f(eps_k) Im G_ij(z_k) on the same layout as G
 * (Eq. EQ-DM-GREEN-FN by quadrature; f(e) = 1/(1+exp((e-mu)/kT)),
 * Eq. EQ-FD-FUNC, evaluated without overflow).
 *   eps, w    host, S doubles: real parts of the shifts and quadrature weights
 *   G         device, n_elem*S complex doubles; rho device, n_elem doubles
 *   stream    cudaStream_t or NULL. Asynchronous on that stream; eps and w
 *             are copied from pageable host memory with cudaMemcpyAsync, so
 *             the call is not meant to be recorded into a CUDA graph (a
 *             captured copy would read the host arrays at replay time). */
int gsk_density(gsk_handle h, int64_t n_elem, int32_t n_shifts, const double* eps,
                const double* w, double mu, double kT, const double* G, double* rho,
                void* stream);

/* Allocation-free variant of gsk_density; the paper has no counterpart.
 *
 * Same result and arguments as gsk_density, but it needs no handle and never
 * allocates device memory. It is meant for callers that cannot call
 * cudaMalloc: applications whose device memory is owned by their own pool
 * allocator, services that forbid allocation after start-up because an
 * allocation can stall the device and has no latency bound, and plug-ins that
 * run inside a host program that hands them buffers but no right to allocate.
 *
 * The shift energies, weights and Fermi-weighted coefficients of a call live
 * in a fixed device array inside libgsk of 3 * GSK_NOALLOC_MAX_SHIFTS doubles
 * (24 KiB). Every GPU that loads the library holds that array until the
 * process exits.
 *   n_shifts  1 .. GSK_NOALLOC_MAX_SHIFTS; larger values return GSK_EINVAL
 *   eps, w    host, n_shifts doubles (copied before the call returns)
 *   G, rho    device buffers on the current device, as for gsk_density
 *   stream    cudaStream_t or NULL; the work is asynchronous on that stream
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the
 * process, so after cudaDeviceReset on a device this entry point must not be
 * called on that device again. All calls share the array: each call
 * overwrites the 3 * n_shifts entries it reads before it reads them, so
 * nothing has to start at zero, but calls whose work overlaps on the GPU
 * (for example on two streams) race on it and must be serialised by the
 * caller. */
#define GSK_NOALLOC_MAX_SHIFTS 1024
int gsk_density_noalloc(int64_t n_elem, int32_t n_shifts, const double* eps, const double* w,
                        double mu, double kT, const double* G, double* rho, void* stream);

/* Tr over the column set of rho X (Eq. TRACE-X restricted to the columns
 * solved): sum_c sum_{t} rho[offsets[c]+t] * X_{cols[c], i_t}, X = A (which=0)
 * or B (which=1). rho device; result written to *out (host). Synchronous. */
int gsk_trace(gsk_handle h, int32_t n_cols, const int32_t* cols, const double* rho,
              int32_t which, double* out);

/* Per-shift traces over the column set (Eq. TRACE-X split by shift):
 *   s[k] = sum_c sum_t Im G[offsets[c]+t][k] * X_{cols[c], i_t},  X = A (which=0) or B (which=1),
 * where i_t runs over P(cols[c]) in G's layout (gsk_pattern_offsets). With
 * them Tr(rho X) = -(1/pi) sum_k w_k f(eps_k) s[k] for any mu and kT, so
 * quantities at several chemical potentials need no second pass over G.
 *   G   device, offsets[n_cols]*n_shifts complex doubles
 *   s   host, n_shifts doubles (written)
 * Synchronous. The order of every sum is fixed (bitwise repeatable). */
int gsk_shift_trace(gsk_handle h, int32_t n_cols, const int32_t* cols, int32_t n_shifts,
                    const double* G, int32_t which, double* s);

/* Chemical potential (Sec. II: mu is set so that the electron count is
 * reproduced): the mu in [mu_lo, mu_hi] with
 *   N(mu) = -(1/pi) sum_k w_k f_mu(eps_k) s_k = n_elec,
 * s_k the per-shift traces with X = B (gsk_shift_trace) and f the Fermi
 * function of Eq. EQ-FD-FUNC with temperature kT. The search runs on the GPU
 * (33-section bracketing, to the resolution of FP64); N(mu_lo) < n_elec <=
 * N(mu_hi) must hold, else GSK_EINVAL (nothing written). If N is not
 * monotone on the bracket (possible for a column subset), the result is one
 * of its roots there.
 *   eps, w  host, n_shifts doubles: Re z_k and quadrature weights
 *   G       device, as for gsk_shift_trace
 *   mu      host out; count host out (N(mu)) or NULL
 * Synchronous. */
int gsk_find_mu(gsk_handle h, int32_t n_cols, const int32_t* cols, int32_t n_shifts,
                const double* eps, const double* w, const double* G, double kT, double n_elec,
                double mu_lo, double mu_hi, double* mu, double* count);

/* The same chemical-potential search from per-shift traces the caller
 * already has (host, n_shifts doubles: s_k with X = B, e.g. gsk_shift_trace
 * results summed over the ranks that share the column set). N(mu), the
 * bracket rule and the outputs are as for gsk_find_mu. Synchronous. */
int gsk_mu_from_traces(gsk_handle h, int32_t n_shifts, const double* eps, const double* w, const double* s,
                       double kT, double n_elec, double mu_lo, double mu_hi, double* mu, double* count);

/* Atom-pair pattern of A in the caller's atom numbering: for atom J,
 * aidx[aptr[J] .. aptr[J+1]) are the atoms I (ascending) with some A_{Ia,Jb}
 * in the pattern, J itself included. aptr: host, n_atoms+1 (written);
 * aidx: host, aptr[n_atoms] entries, or NULL to query the size first. */
int gsk_atom_pattern(gsk_handle h, int64_t* aptr, int32_t* aidx);

/* Connectivity matrix (Sec. VII, the integrated crystal orbital Hamiltonian
 * population): C_IJ = sum_a sum_b rho_{Ia;Jb} A_{Jb;Ia}, summed over the
 * solved columns Jb in cols only, on the atom pattern of gsk_atom_pattern:
 * C[aptr[J] + s] = C_{aidx[s], J}. Slots of atoms without a column in cols
 * are 0. Summing C gives Tr(rho A) over the same columns (the electronic
 * energy when cols covers every row).
 *   rho   device, laid out like G without the shift axis (gsk_density's output)
 *   C     device, aptr[n_atoms] doubles (written)
 *   stream  cudaStream_t or NULL; the gather lists are copied before the
 *           call returns and the kernel runs asynchronously on that stream.
 * Each slot sums its terms in a fixed order (bitwise repeatable). */
int gsk_icohp(gsk_handle h, int32_t n_cols, const int32_t* cols, const double* rho, double* C,
              void* stream);

/* Multiple Arnoldi projection (Sec. III-B, Eq. EQ-LS-MULTIPLE,
 * EQ-EIG-GREEN-KRYLOV, EQ-PROJ-PHYS-QUANT-KRYLOV): for each column j the
 * pencil is projected onto K_{nu/2}(A; e_j) + K_{nu/2}(A; B^-1 e_j); the
 * reduced problem gives Ritz values eps_m and B-orthonormal Ritz vectors v_m,
 * and the energy integral is done analytically:
 *   rho_ij    = sum_m f(eps_m) (v_m)_i (v_m)_j                 i in P(j)
 *   G_ij(z_k) = sum_m (v_m)_i (v_m)_j / (z_k - eps_m)           (optional)
 * This is the paper's own approximation, not the exact-to-tolerance solve
 * of gsk_solve: it is exact when nu/2 reaches the dimension of the Krylov
 * space of e_j. Directions of the second subspace within sin(theta) < 1e-7 of
 * the first are dropped, and a Krylov sequence ends early where it becomes
 * invariant (new direction below 1e-13 ||A||_inf), so the rank r can be
 * below nu.
 *   nu       even, 2 .. GSK_MA_MAX_NU
 *   mu, kT   Fermi function of Eq. EQ-FD-FUNC (kT > 0)
 *   rho      device, offsets[n_cols] doubles, G's layout without the shift axis
 *   n_shifts 0, or S >= 1 with z (host, 2*S doubles: re, im) and G (device,
 *            offsets[n_cols]*S complex doubles, as for gsk_solve)
 *   ritz     host, n_cols*nu doubles or NULL: eps_m ascending, NaN past r
 *   weight   host, n_cols*nu doubles or NULL: (v_m)_j^2 (rho_jj = sum f w)
 *   charge   host, n_cols*nu doubles or NULL: (v_m)_j (B v_m)_j; their sum
 *            is 1 for every column (e_j lies in the subspace)
 *   rank     host, n_cols or NULL: r, or -1 if Q^T B Q was not positive
 *            definite (the column's outputs are then not meaningful)
 * Columns run in batches of 32 on FP64 arithmetic. Synchronous. Returns
 * GSK_ETIMEOUT if the CG for B^-1 e_j did not reach 1e-15 in 2000 steps. */
#define GSK_MA_MAX_NU 32
int gsk_marnoldi(gsk_handle h, int32_t n_cols, const int32_t* cols, int32_t nu, double mu, double kT,
                 double* rho, int32_t n_shifts, const double* z, double* G, double* ritz, double* weight,
                 double* charge, int32_t* rank);

/* Real-space projection (Sec. III-B): column j is solved on the pencil
 * restricted to the orbitals of the region around its atom J -- every atom
 * within the distance of J's kappa-th nearest atom (J counted, ties kept),
 * so the region holds kappa atoms or more -- by the multiple Arnoldi
 * projection of gsk_marnoldi (same nu, mu, kT, outputs and conventions, with
 * ritz/weight/charge/rank of the projected problem). Distances use the
 * positions given to gsk_create (required; GSK_EINVAL without them) and the
 * minimum-image convention in the periodic box (Lx, Ly, Lz) when box is not
 * NULL.
 *   rho      device, the layout of gsk_pattern_offsets without the shift
 *            axis; entries whose row lies outside the region are 0
 *   m_local  host, n_cols or NULL: orbitals in each column's region (M')
 * The regions are found and the restricted pencils assembled on the host
 * (a batch of 32 columns becomes one block-diagonal pencil solved on the
 * GPU). On first use the matrix values are copied back to the host once.
 * Synchronous. */
int gsk_marnoldi_projected(gsk_handle h, const double* box, int32_t kappa, int32_t n_cols, const int32_t* cols,
                           int32_t nu, double mu, double kT, double* rho, double* ritz, double* weight,
                           double* charge, int32_t* rank, int32_t* m_local);

/* Library row order: row_lib[i] = row of caller row i in the layout used by
 * gsk_spmm (host array of M entries). */
int gsk_row_order(gsk_handle h, int32_t* row_lib);

/* n_rep applications of the solver's block SpMM kernel, Y = S X with S = A
 * (which = 0) or B (which = 1 or 2), on W lanes (32, 64 or 128; 128 only for
 * FP32): the same kernel, launch shape and epilogue that gsk_solve runs, for
 * timing and for callers working in the library's row order. For B it is the
 * inner CG's kernel, which also sets a direction vector P = X (internal) and
 * forms the per-lane dot P.Y; for A it forms the dot X.Y. For B, which = 1
 * runs the per-atom gather kernel and which = 2 the staged kernel
 * (GSK_MIXED only; it returns GSK_ETIMEOUT if one of its bounded waits gave
 * up).
 *   precision GSK_FP64: X, Y are double; GSK_MIXED: X, Y are float
 *   X, Y      device, M x W row-major (lane fastest), rows in library order
 *   stream    cudaStream_t or NULL. Asynchronous on that stream. */
int gsk_spmm(gsk_handle h, int32_t which, int32_t precision, int32_t W, const void* X, void* Y,
             int32_t n_rep, void* stream);

/* ----- learned column scheduler ---------------------------------------------
 * A 16 -> 64 -> 64 -> 1 multilayer perceptron (tanh, FP32) predicts log(number
 * of Lanczos steps) of a column from 16 per-column features; with
 * sched = GSK_SCHED_LEARNED, gsk_solve hands out columns longest predicted
 * first, which shortens the tail of the work queue (the load imbalance from
 * structural disorder of Sec. IV-C). Every column still iterates to tol.
 * Parameters: one flat FP32 vector W1 [64][16], b1 [64], W2 [64][64], b2 [64],
 * w3 [64], b3 [1]. Normalisation: 32 floats, mean[16] then std[16] (> 0);
 * the network sees (feature - mean) / std. Features of column j = (atom J,
 * orbital a) with damping eta: log(eta), 0.1/eta, entries of row j / 100,
 * neighbour atoms of J / 50, 4-orbital neighbours / 20, 1-orbital neighbours
 * / 40, [J has 4 orbitals], a/3, A_jj/10, sum_{i!=j}|A_ij|/10,
 * sum_{i!=j}|B_ij|, sqrt(sum_{i!=j} A_ij^2)/10, A_jj^2/100, B_jj,
 * log(1 + sum_i |A_ij|), 1. */
#define GSK_MLP_IN 16
#define GSK_MLP_HIDDEN 64
#define GSK_MLP_NPARAM 5313

/* Features of columns cols[0..n) with dampings eta (host arrays) into feat
 * (device, n x 16 row-major). Synchronous. */
int gsk_features(gsk_handle h, int32_t n_cols, const int32_t* cols, const double* eta, float* feat,
                 void* stream);

/* y[s] = MLP(params, (feat[s] - mean) / std) for n samples (all device
 * pointers, current device). Asynchronous on stream. */
int gsk_mlp_forward(int32_t n, const float* feat, const float* norm, const float* params, float* y,
                    void* stream);

/* Bytes of the device workspace gsk_mlp_train_step needs for n samples. */
size_t gsk_mlp_workspace_bytes(int32_t n);

/* One full-batch step on the mean squared error (1/n) sum (y - target)^2:
 * gradient by backpropagation (deterministic fixed-order sums), then, if
 * t >= 1, one Adam update (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias
 * correction with step number t). grad (n_param floats) and loss (1 float,
 * the loss before the update) are optional outputs. All pointers device;
 * work holds gsk_mlp_workspace_bytes(n) bytes. Asynchronous on stream. */
int gsk_mlp_train_step(int32_t n, const float* feat, const float* norm, const float* target, float* params,
                       float* adam_m, float* adam_v, int32_t t, float lr, float* grad, float* loss,
                       void* work, void* stream);

/* Install a trained model (host arrays) on the handle for GSK_SCHED_LEARNED. */
int gsk_set_sched_model(gsk_handle h, const float* params, const float* norm);

/* Autotuner of the lane width W (columns in flight) and, in the mixed modes,
 * of the inner-CG product kernel. For each candidate W (32, 64 and, in the
 * mixed modes, 128) and kernel (GSK_SPMM_GATHER, and GSK_SPMM_STAGED in the
 * mixed modes) it times, with CUDA events, a truncated solve (24 Lanczos
 * steps) of the first columns of the set and picks the pair that minimises
 * the estimated time of the whole set, t_step * max(n_cols / W, 2) in units
 * of a column's mean step count (the factor 2 accounts for the longest column
 * of a set with mixed damping). The result is kept on the handle for
 * opt->precision (and the best kernel for every W measured) and used by
 * gsk_solve whenever opt->batch_w or opt->spmm_kernel is 0. If the
 * environment variable GSK_TUNE_CACHE names a file, results are cached there
 * across processes, one line per (M, nnz, atoms, precision, shifts, columns,
 * GPU name, SM count): a hit skips the measurement; a miss appends a line.
 * Arguments as for gsk_solve; *best_w receives the W chosen (host).
 * Synchronous. */
int gsk_autotune(gsk_handle h, int32_t n_shifts, const double* z, const double* eta, int32_t n_cols,
                 const int32_t* cols, const gsk_options* opt, int32_t* best_w);

/* The last gsk_autotune result for a precision mode (host outputs, each may
 * be NULL): the W and kernel chosen, whether they came from the cache file,
 * and the candidates measured (up to 8: W, kernel, milliseconds per lock-step
 * Lanczos step; none on a cache hit). */
int gsk_autotune_result(gsk_handle h, int32_t precision, int32_t* w, int32_t* kernel, int32_t* from_cache,
                        int32_t* n_cand, int32_t* cand_w, int32_t* cand_kernel, double* cand_ms_per_step);

/* Measured FMA throughput of the current device, for the roofline of the
 * ALU-bound kernels (the FP64 block products of gsk_marnoldi): every thread
 * runs 8 or 16 independent FMA chains over a grid of 8 CTAs per SM; *tflops
 * (host) receives the best of 2 * n_rep timed launches (CUDA events on
 * stream, after one untimed launch) in TFLOP/s, 2 flops per FMA. precision: GSK_FP64 or
 * GSK_MIXED (FP32). Allocates a small device buffer for the chains' results.
 * Synchronous. The paper has no counterpart: it is a measurement tool. */
int gsk_alu_peak(int32_t precision, int32_t n_rep, double* tflops, void* stream);

/* Counters of the last gsk_solve on this handle. */
typedef struct {
  int64_t outer_steps;       /* Lanczos steps of the lane batch (lock-step) */
  int64_t cg_iterations;     /* inner CG iterations, all B-solve passes */
  int64_t kernel_launches;   /* kernels the solve launched (graph nodes executed) */
  int32_t batch_w;           /* lanes used */
  int32_t used_graph;        /* 1 when the solve ran as one CUDA graph */
  int32_t spmm_kernel;       /* GSK_SPMM_GATHER or GSK_SPMM_STAGED: kernel of the inner-CG products */
  int32_t debug_code;        /* bounds-checked build: first failed index check of the last gsk_solve or
                                gsk_spmm (a code listed at the top of this file), 0 = none; always 0 otherwise */
  int64_t debug_index;       /* the index that failed it */
} gsk_stats;

/* Copy the counters of the last gsk_solve into *out (host). */
int gsk_last_stats(gsk_handle h, gsk_stats* out);

/* Human-readable text for a GSK_* code. */
const char* gsk_strerror(int code);

/* Bounds-checked build: runs one kernel whose index check fails on purpose
 * (it guards no memory access) and reads the record back: *code (host) = 99,
 * *index (host) = 12345678901 when the recording path works; the record is
 * cleared again. Synchronous, on the legacy default stream, no handle. The
 * normal build returns GSK_ENOTSUP with *code = *index = 0. A test utility
 * of the library; the paper has no counterpart. */
int gsk_debug_selftest(int32_t* code, int64_t* index);

#ifdef __cplusplus
}
#endif

#endif /* GSK_H */
