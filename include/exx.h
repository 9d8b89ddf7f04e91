/*
 * exx.h -- C interface of the GB300 exact-exchange library (libexx_gb300.so).
 *
 * The library applies the exact-exchange operator of a hybrid functional on a
 * real-space finite-difference grid and builds the adaptively compressed exchange
 * (ACE) operator from it, following "GPU acceleration of hybrid functional
 * calculations in the SPARC electronic structure code" (arXiv 2501.16572):
 *   - exchange operator, Eq. 1 (Gamma point, real orbitals, one spin channel);
 *   - pair Poisson problems, Eq. 2 (unscreened) and Eq. 3 (erfc-screened);
 *   - their solution X = f(L) B through the Kronecker eigen-decomposition of the
 *     finite-difference Laplacian, Eqs. 4-7, solved as a batch (Sec. II.B);
 *   - ACE construction, Sec. III.A: W, M = Psi^T W, Cholesky factor, xi.
 *
 * Conventions shared by every call
 *   Grid:     N = Nx*Ny*Nz points, spacing h (bohr), index r = ix + Nx*(iy + Ny*iz)
 *             (x fastest).  dV = h^3.
 *   Orbitals: real FP64, column-major N x n blocks with leading dimension ld >= N;
 *             column j starts at base + j*ld.  Orbitals are expected to be
 *             orthonormal in the dV metric, sum_r psi_m psi_n dV = delta_mn (only
 *             ACE needs this; exx_apply works for any input).
 *   Memory:   every array pointer is a DEVICE pointer owned by the caller (for
 *             example a PyTorch tensor) unless the name ends in _h; the library
 *             never frees or keeps caller memory.  The plan owns its own device
 *             workspace.  Arrays must be 8-byte aligned; a call does not modify
 *             its inputs.
 *   Streams:  calls are asynchronous on `stream` (NULL = legacy default stream)
 *             unless stated otherwise.  One plan must not be used by two calls
 *             that overlap in time (it owns one workspace).
 *   Errors:   every call returns an exx_status; nothing throws across the
 *             interface.  Arguments are checked on the host before any launch;
 *             a failing CUDA call is reported as EXX_ERR_CUDA and its text is kept
 *             for exx_last_error().
 *   Device:   compiled for sm_103a (GB300).  There is no CPU fallback: without a
 *             usable GPU every compute call returns EXX_ERR_CUDA.
 */
#ifndef EXX_GB300_H
#define EXX_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct exx_plan_s *exx_plan;
/* Same type as cudaStream_t; declared here so this header needs no CUDA include. */
typedef struct CUstream_st *exx_stream_t;

typedef enum {
    EXX_OK = 0,
    EXX_ERR_INVALID_ARG = 1,   /* bad size, pointer, enum or leading dimension */
    EXX_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed */
    EXX_ERR_OOM = 3,           /* device workspace could not be allocated */
    EXX_ERR_NOT_POSDEF = 4,    /* ace_build: -sym(M) is not positive definite */
    EXX_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    EXX_ERR_UNSUPPORTED = 6    /* valid but unsupported combination */
} exx_status;

enum { EXX_BC_DIRICHLET = 0, EXX_BC_PERIODIC = 1 };

/* Kernels f of Eq. 5, on the eigenvalues lambda <= 0 of the FD Laplacian:
 *   COULOMB             f = -4 pi / lambda                         (Eq. 2)
 *   ERFC                f = 4 pi/|lambda| (1 - exp(-|lambda|/(4 omega^2))), f(0) = pi/omega^2
 *                       (erfc-screened HSE kernel; Eq. 3 as printed has an exponent
 *                       that grows without bound, this is the reading used)
 *   ERFC_PAPER16PI      same with 16 pi omega^2 in place of 4 omega^2 (the printed
 *                       magnitude), kept only for comparison. */
enum { EXX_KERNEL_COULOMB = 0, EXX_KERNEL_ERFC = 1, EXX_KERNEL_ERFC_PAPER16PI = 2 };

/* Arithmetic of the mode products (the six contractions of the batched Kronecker
 * solve, Sec. II.B):
 *   FP64     double precision on the CUDA cores;
 *   BF16X3   tcgen05 tensor cores; every row is scaled by a power of two and cut into
 *            two 8-bit fixed-point slices stored as bf16; the 3 slice products of
 *            levels 0-1 are summed exactly (one FP32 TMEM accumulator per level, every
 *            partial sum an integer below 2^24); ~16 bits;
 *   BF16X6   as BF16X3 with three data slices (6 products, levels 0-2) and a fourth
 *            slice of the shared eigenvector matrices used against the leading data
 *            slice; ~24 bits, FP32 intermediates between passes;
 *   BF16X10  four slices per operand (10 products, levels 0-3) and intermediates kept
 *            as hi+lo FP32 pairs between passes; ~32 bits;
 *   TF32X3   floating tf32 split, 3 products into one FP32 accumulator (the tensor core
 *            rounds that accumulation toward zero, a bias common to all pairs); kept
 *            for comparison.
 *   BF16X7   three passes over HBM instead of five (x and y products per z-slice with
 *            the tile transposed on chip; z forward, f(Lambda) and z inverse per pencil),
 *            FP32 intermediates; base-512 digits: three per data row, four per matrix row;
 *            the leading product summed exactly in one TMEM accumulator, the six others
 *            in a second; the fully modal middle kept as FP32 hi + lo; ~27 bits per
 *            product.  Needs Nx, Ny <= 128 (EXX_ERR_UNSUPPORTED otherwise) and up to
 *            about 208 points along z; matrices too large to stay in shared memory (the
 *            z matrices of long axes, the x/y matrices of slices wider than about 108
 *            points) stream through it as K-chunks.
 * Pair densities and the accumulation over pairs are compensated in every mode. */
enum { EXX_PREC_FP64 = 0, EXX_PREC_BF16X3 = 1, EXX_PREC_TF32X3 = 2, EXX_PREC_BF16X6 = 3,
       EXX_PREC_BF16X10 = 4, EXX_PREC_BF16X7 = 5 };

/* Create a plan for one grid (Sec. II.A, Eqs. 6-7).  Host FP64 work, done once:
 * FD weights of order fd_order (even, 2..24), the three 1D second-derivative
 * operators (Dirichlet: zero outside the grid; periodic: circulant), their
 * eigen-decompositions, f over the eigenvalue sums; the results are uploaded to
 * the device.  Nx, Ny, Nz in [2, 256]; h > 0; bc[d] in {DIRICHLET, PERIODIC};
 * omega > 0 for the ERFC kernels.  COULOMB with all three axes periodic has a
 * zero eigenvalue and returns EXX_ERR_UNSUPPORTED.  Uses the current CUDA device.
 * On success *out is a new plan (free with exx_plan_destroy). */
int exx_plan_create(exx_plan *out, int Nx, int Ny, int Nz, double h, const int bc[3],
                    int fd_order, int kernel, double omega);

/* Select the mode-product arithmetic (EXX_PREC_*); default EXX_PREC_FP64.  The split
 * modes upload fixed-point images of the 1D eigenvector matrices; an axis whose images
 * do not fit in one CTA's shared memory is cut into blocks of ceil(n/nb) points (nb <= 16)
 * and each mode product becomes nb x nb block products summed in hi/lo FP32
 * (EXX_ERR_UNSUPPORTED if 16 blocks do not fit). */
int exx_plan_set_precision(exx_plan plan, int prec);

/* Tuning: pairs per batch (the paper's n_c, Sec. II.B) and orbitals per pair block.
 * 0 = defaults: blocks of 8 orbitals, and as many pairs per batch as fit two plan-owned
 * work buffers of at most 2 GiB each, at most 1024, a multiple of block^2.  Results do
 * not depend on either (up to the order of the compensated sums). */
int exx_plan_set_batch(exx_plan plan, int pairs_per_batch, int block_orbitals);

/* Shard the pair solves of exx_apply over `world` processes (one GPU each): this plan then
 * runs only the batches b with b mod world == rank and writes PARTIAL outputs; summing
 * `out` over the ranks (one all-reduce or reduce-scatter of N x n_in doubles) gives the
 * full result.  Each unique pair is solved by exactly one rank.  world = 1 (default)
 * runs everything.  0 <= rank < world. */
int exx_plan_set_shard(exx_plan plan, int rank, int world);

/* Autotuner of the tile and schedule settings (Sec. II.B's batch size n_c and the kernel
 * shapes), measured on this grid with the caller's own data: exx_apply's arguments and
 * rules (out is used as scratch and left holding partial results).  Coordinate descent over
 *   pairs per batch {default, 256, 512, 1024} x orbitals per pair block {8, 16}, then, in
 *   the BF16X7 mode, the pass-B matrix streaming (output blocks or K-chunks, their width
 *   and shared-memory buffer count: every choice that fits), then the slice passes' form (serial with up to two CTAs per SM, or
 *   software-pipelined over tiles with one CTA per SM) with their input staging (auto, off, on);
 * each candidate runs up to three batches of the pair schedule twice (warm-up, then timed
 * with CUDA events on `stream`); the fastest per pair solve is kept in the plan (as by
 * exx_plan_set_batch) and in a process-wide cache keyed by grid, boundary conditions,
 * precision, n_occ, n_in and aliasing, so that a later plan with the same key takes it
 * without measuring.  flags bit 0 = measure again even if cached.  Synchronizes `stream`.
 * Results of exx_apply do not depend on the choice (up to the order of compensated sums). */
int exx_plan_autotune(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
                      const double *Psi_in, int n_in, long ld_in, double *out, long ld_out, int flags,
                      exx_stream_t stream);

/* The plan's settings (HOST int[6]: pairs per batch, orbitals per block, pass-B block width
 * (> 0: output blocks of that many columns; < 0: K-chunks of that many contraction indices),
 * pass-B buffers, slice staging, slice pipeline; 0 / -1 = automatic), the autotuner's trial time per pair
 * solve in ms (0 if never tuned) and *tuned_h = 0 (not tuned), 1 (measured), 2 (cache). */
int exx_plan_get_tuning(exx_plan plan, int *settings_h, double *ms_per_pair_h, int *tuned_h);

/* Set the same six settings by hand (for instance a choice the autotuner made earlier):
 * pairs per batch >= 0, block in [0, 32], pass-B block width (|width| a multiple of 16,
 * <= 256; negative = K-chunks) and
 * buffers (both 0 = automatic, or both set; a pair that does not fit falls back to the
 * automatic choice), staging and pipeline in {-1, 0, 1}.  EXX_ERR_INVALID_ARG otherwise. */
int exx_plan_set_tuning(exx_plan plan, const int *settings_h);

/* Free the plan and its device workspace (synchronizes the device first). */
int exx_plan_destroy(exx_plan plan);

/* Copy plan data to HOST memory for inspection: which = 0,1,2 gives the eigenvalues
 * of axis d (n_d values); which = 3 gives f(Lambda) (N values, index
 * a + Nx*(b + Ny*c)).  `count` must equal the number of values. */
int exx_plan_get(exx_plan plan, int which, double *dst_h, long count);

/* Exact-exchange operator, Eq. 1 (and Eq. W of Sec. III.A):
 *   out_n = - sum_{m < n_occ} f_m psi_m (.) phi_mn,  phi_mn = f(L)(psi_m (.) psi_n)
 * for n = 0..n_in-1, where psi_m are the columns of Psi_occ and psi_n those of Psi_in.
 * Psi_occ: N x n_occ (ld_occ), f: n_occ device doubles, Psi_in: N x n_in (ld_in),
 * out: N x n_in (ld_out), overwritten.  out must not overlap the inputs.
 * When Psi_in == Psi_occ and ld_in == ld_occ (the ACE case: n_in >= n_occ, the
 * occupied orbitals leading), each pair among the occupied orbitals is solved once
 * and used for both out_m and out_n (phi_mn = phi_nm).  1 <= n_occ, n_in <= 65536. */
int exx_apply(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
              const double *Psi_in, int n_in, long ld_in, double *out, long ld_out,
              exx_stream_t stream);

/* The original (non-batched) Kronecker product formalism of Sec. II.A, Eq. 8: the same
 * result as exx_apply (same arguments, layout, aliasing rule and errors), computed in FP64
 * whatever the plan's precision, one orbital pair at a time, each pair's linear system with
 * its 4 n_z + 2 dense matrix products issued as separate small GEMM launches (per frontal
 * slice Vx^T B_k Vy, then the z axis, the f(Lambda) product, and the inverse).  It is there
 * to measure what batching the right-hand sides buys (Sec. II.B, Figs. 1-2); it is launch
 * bound by design and far slower than exx_apply.  Needs 3 N doubles of plan workspace. */
int exx_apply_original(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
                       const double *Psi_in, int n_in, long ld_in, double *out, long ld_out,
                       exx_stream_t stream);

/* Exchange energy E_x = 1/4 sum_{n < n_occ} f_n dV <psi_n, VxPsi_n>, FP64 with
 * compensated (Neumaier) sums in a fixed order (the paper prints no formula; this
 * is the spin-unpolarised Fock energy for occupations f in [0, 2]).  Writes the
 * HOST double *E_x_h; synchronizes `stream`. */
int exx_energy(exx_plan plan, const double *Psi_occ, int n_occ, long ld, const double *f,
               const double *VxPsi, long ld_v, double *E_x_h, exx_stream_t stream);

/* ACE construction, Sec. III.A:
 *   M = dV Psi^T W (n x n),  -sym(M) = L L^T (L lower triangular, positive diagonal),
 *   xi = W L^{-T} (N x n).
 * The compressed operator is then -dV xi xi^T (M is negative definite, so the
 * printed "Cholesky factor of M" is read as that of -M).  Psi, W: N x n (ld, ld_w);
 * xi: N x n (ld_xi), overwritten; M_out: optional n x n column-major device buffer
 * (NULL to skip).  FP64 plans compute every step on the CUDA cores in FP64.  Split
 * plans compute the products M and xi on the tensor cores: fixed-point digits of 31
 * bits per 320-long chunk of the contraction (rows scaled by their largest entry),
 * exact integer sums per chunk, FP64 across chunks (relative error ~1e-9..1e-8).  The
 * Cholesky factor and its inverse are FP64 in every mode.
 * *info_h (host) is 0, or 1 + the failing pivot when EXX_ERR_NOT_POSDEF is
 * returned.  Synchronizes `stream`.  n <= 2048. */
int ace_build(exx_plan plan, const double *Psi, int n, long ld, const double *W, long ld_w,
              double *xi, long ld_xi, double *M_out, int *info_h, exx_stream_t stream);

/* ACE application, Sec. III.B: out = -dV xi (xi^T Phi); xi: N x n, Phi, out: N x nphi.
 * Both products run as in ace_build: FP64 for FP64 plans, tensor-core digits for split
 * plans. */
int ace_apply(exx_plan plan, const double *xi, int n, long ld_xi, const double *Phi, int nphi,
              long ld_phi, double *out, long ld_out, exx_stream_t stream);

/* One ACE outer step from HOST buffers: copies Psi_h (N x n, ld) and f_h (n_occ) to
 * plan-owned device buffers, runs exx_apply (Psi_occ = the first n_occ columns,
 * Psi_in = all n), exx_energy and ace_build, and copies xi back to xi_h (N x n,
 * ld_xi) and the energy to *E_x_h.  Synchronous. */
int exx_ace_step_host(exx_plan plan, const double *Psi_h, int n, long ld, int n_occ,
                      const double *f_h, double *xi_h, long ld_xi, double *E_x_h, int *info_h,
                      exx_stream_t stream);

/* Many independent systems in one call: the batching of Sec. II.B carried across
 * systems (for instance 48 small molecules of different grids and orbital counts).
 * For each s < nsys the result in args[s].out equals what exx_apply(plans[s],
 * args[s]...) writes, bit for bit; args[s] has exx_apply's meaning, layout and rules.
 *   1. Every system is checked and every device allocation is made first (this
 *      synchronizes `stream` when a plan's pair schedule has to be rebuilt).
 *   2. On a stream other than NULL, with timing off on every plan, the launches of
 *      all systems are captured once into one CUDA graph (relaxed capture mode), the
 *      systems spread over 8 concurrent branches (system s on branch s mod 8, forked from
 *      and joined back into `stream`) so that small systems share the GPU, and kept in a
 *      library-wide cache of 8 graphs, keyed by the plans, their settings
 *      and every pointer, size and leading dimension in args; a later call with the
 *      same key replays the graph: one launch from the host for the whole sequence.
 *      A replay reads whatever the pointed-to buffers hold at that time, so callers
 *      refill the same buffers in place between calls.
 *   3. With stream NULL, or timing on, the launches are issued one by one.
 * Every plan must use the same precision and appear at most once in plans[] (a plan owns
 * one pair schedule and one workspace; a repeated plan returns EXX_ERR_INVALID_ARG before
 * anything runs); a plan must not be used by another call on another stream while its
 * work is in flight.  exx_plan_destroy drops the cached
 * graphs that use the plan.  Errors: EXX_ERR_INVALID_ARG (NULL or inconsistent
 * arguments, with the index-free message of exx_apply), EXX_ERR_OOM, EXX_ERR_CUDA
 * (capture, instantiation or launch failed). */
typedef struct {
    const double *Psi_occ; int n_occ; long ld_occ; const double *f;
    const double *Psi_in; int n_in; long ld_in; double *out; long ld_out;
} exx_apply_args;
int exx_apply_batched(const exx_plan *plans, int nsys, const exx_apply_args *args,
                      exx_stream_t stream);

/* Number of kernel launches issued by the last exx_apply / ace_build / energy call
 * on this plan (for benchmarks). */
long exx_plan_launch_count(exx_plan plan);

/* Per-kernel timing with CUDA events recorded on the launch stream around every
 * kernel the plan launches (for benchmarks).  enable = 1 starts recording (and clears
 * earlier records), 0 stops.  exx_plan_get_timing synchronizes the device and returns,
 * for kernel class `kind` (EXX_TIMING_*), the summed device time in milliseconds and
 * the number of launches recorded since timing was enabled. */
enum { EXX_TIMING_PASS1 = 0, EXX_TIMING_PASS2 = 1, EXX_TIMING_PASS3 = 2, EXX_TIMING_PASS4 = 3,
       EXX_TIMING_PASS5 = 4, EXX_TIMING_ACCUM = 5, EXX_TIMING_PREP = 6, EXX_TIMING_GEMM = 7,
       EXX_TIMING_CHOL = 8, EXX_TIMING_ENERGY = 9, EXX_TIMING_KINDS = 10 };
int exx_plan_set_timing(exx_plan plan, int enable);
int exx_plan_get_timing(exx_plan plan, int kind, double *ms_h, long *launches_h);

/* Gram matrix M = dV Psi^T W (n x n, column-major, written to the DEVICE buffer M)
 * without any device allocation.  This entry point has no counterpart in the paper; it
 * serves callers that cannot call cudaMalloc when they need M: programs whose device
 * memory belongs to a pool or framework allocator this library cannot use, processes
 * that reserve all device memory up front, and loops that must not stall (cudaMalloc and
 * cudaFree can synchronize the whole device).  It needs no plan.  Psi, W: N x n DEVICE blocks (ld, ld_w >= N), n in [1, 128]; larger n
 * returns EXX_ERR_INVALID_ARG and launches nothing.  The split-K partial sums go to a
 * fixed 1 MiB device array inside the library (one per GPU that loads it, kept until
 * the process exits).  The first call on each device looks up that array's address with
 * the device current, so make that first call before any stream capture.  Every call
 * rewrites all of the array it reads, so no clearing is needed, but all calls share the
 * one array: calls that overlap on the GPU (different streams, or different host
 * threads) race and must be serialised by the caller.  Asynchronous on `stream`. */
int exx_gram_noalloc(int N, double dV, const double *Psi, int n, long ld, const double *W, long ld_w,
                     double *M, exx_stream_t stream);

/* ---- Complex (Bloch) path: Eq. 1 with Brillouin-zone wavevectors --------------------------
 * The pair problems of Eqs. 2-3 for rho = conj(psi_{m q}) phi_{n k} are solved with Bloch
 * boundary conditions at k - q along the periodic axes and Dirichlet conditions along the
 * others (Sec. II, below Eq. 3), FP64 on the CUDA cores.  Complex arrays are interleaved
 * (re, im) doubles; orbital blocks are N x n complex, column-major, leading dimensions
 * counted in complex elements.  Grids of at most 2^20 points.
 *
 * exx_plan_create_bloch: as exx_plan_create, plus theta[3], the Bloch phase across one
 * period of each axis (theta_d = (k - q)_d L_d; ignored on Dirichlet axes).  Periodic axes use
 * the plane-wave eigenbases u_p(j) = exp(i phi_p j)/sqrt(n), phi_p = (2 pi p + theta)/n, with
 * eigenvalues (w0 + 2 sum_k w_k cos(k phi_p))/h^2.  COULOMB is UNSUPPORTED only when every
 * axis is periodic and every theta is 0 (mod 2 pi).  The plan serves only the calls below. */
int exx_plan_create_bloch(exx_plan *out, int Nx, int Ny, int Nz, double h, const int bc[3],
                          int fd_order, int kernel, double omega, const double theta[3]);

/* One q-term of Eq. 1 for the plan's k - q:
 *   out_n (+)= - sum_{m < n_occ} f_m psi_m (.) phi_mn,  phi_mn = f(L_{k-q}) (conj(psi_m) (.) psi_n),
 * psi_m = columns of Psi_occ (orbitals at q, weights f_m = w_q g_{m q}, device doubles),
 * psi_n = columns of Psi_in (functions at k).  accumulate = 0 overwrites out, 1 adds to it
 * (sum the q-terms with one Bloch plan per k - q).  Every ordered pair is solved. */
int exx_apply_complex(exx_plan plan, const double *Psi_occ, int n_occ, long ld_occ, const double *f,
                      const double *Psi_in, int n_in, long ld_in, double *out, long ld_out,
                      int accumulate, exx_stream_t stream);

/* E = 1/4 sum_n f_n dV Re <psi_n, VxPsi_n> (HOST *E_x_h; synchronizes `stream`). */
int exx_energy_complex(exx_plan plan, const double *Psi, int n, long ld, const double *f,
                       const double *VxPsi, long ld_v, double *E_x_h, exx_stream_t stream);

/* Complex ACE (Sec. III.A): M = dV Psi^H W, -(M + M^H)/2 = L L^H, xi = W L^{-H}; the
 * compressed operator is -dV xi xi^H.  n <= 96 (one-CTA Cholesky).  *info_h = 0 or 1 + the
 * failing pivot with EXX_ERR_NOT_POSDEF.  Synchronizes `stream`. */
int ace_build_complex(exx_plan plan, const double *Psi, int n, long ld, const double *W, long ld_w,
                      double *xi, long ld_xi, int *info_h, exx_stream_t stream);

/* out = -dV xi (xi^H Phi). */
int ace_apply_complex(exx_plan plan, const double *xi, int n, long ld_xi, const double *Phi, int nphi,
                      long ld_phi, double *out, long ld_out, exx_stream_t stream);

/* Static text for a status code; never NULL. */
const char *exx_status_string(int status);

/* Text of the last error recorded by this thread (empty when none). */
const char *exx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EXX_GB300_H */
