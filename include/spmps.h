/*
 * spmps.h -- C ABI of the GB300 (sm_103a) library for spin-projected matrix product states.
 *
 * The library optimises an MPS |Psi> with good particle number N and spin projection M
 * (Abelian (N, M) block sparsity) for the spin-projected energy functional
 *     E = <Psi| H P |Psi> / <Psi| P |Psi>,     P = sum_g c_g exp(-i beta_g S_y)
 * (Li & Chan, arXiv 1703.04789, Eq. efunctional and Eq. pmpo; c_g = (2S+1)/2 w_g d^S_MM(beta_g)
 * with Gauss-Legendre weights w_g in x = cos(beta)).  Every contraction runs in the library's
 * CUDA kernels; there is no CPU fallback: without a usable sm_103a device every entry point
 * that needs one returns SPMPS_ERR_CUDA.
 *
 * Conventions shared by all entry points
 *   - Sites are spatial orbitals k = 0 .. K-1 (Sec. 2.1, last paragraph).  The local basis of a
 *     site is {|0>, |b>, |a>, |ab>}, index 2*n_alpha + n_beta, |ab> = a+_alpha a+_beta |0>, with
 *     Jordan-Wigner order alpha before beta on each site (Eq. JWtrans merged per site).
 *   - Bond i (0..K) carries the quantum numbers (n, 2m) accumulated over sites 0..i-1.  Its
 *     indices are sorted by (n, 2m); the indices of one label are contiguous.
 *   - Two-site tensors x, y, z at sites (k, k+1) use the "row-block layout": for each label
 *     lambda_a of bond k in bond order, one dense row-major block of dim(lambda_a) rows and
 *     W(lambda_a) columns; the columns run over s = 4*s1 + s2 ascending and, inside s, over the
 *     indices of the label lambda_a + q(s1) + q(s2) of bond k+2 (absent labels contribute no
 *     columns).  spmps_x_layout() returns the block table.  Entries outside the (N, M)
 *     pattern do not exist in this layout.
 *   - Handles own all device memory they use.  Host arrays passed in are copied; the caller
 *     keeps ownership.  No C++ exception crosses this interface.
 *   - Thread safety: one handle must not be used from two threads at once.
 */
#ifndef SPMPS_H
#define SPMPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmps_t* spmps_handle;

typedef enum {
    SPMPS_OK = 0,
    SPMPS_ERR_BAD_INPUT = 1,        /* invalid argument; no device work was done          */
    SPMPS_ERR_NOT_CONVERGED = 2,    /* an iteration hit its cap; best result kept          */
    SPMPS_ERR_SINGULAR_METRIC = 3,  /* the projected norm matrix has no usable range       */
    SPMPS_ERR_OOM = 4,              /* device allocation failed                            */
    SPMPS_ERR_TIMEOUT = 5,          /* a bounded device wait gave up                       */
    SPMPS_ERR_CUDA = 6,             /* CUDA runtime error (message in spmps_last_error)    */
    SPMPS_ERR_NAN = 7,              /* NaN or Inf detected in a result                     */
    SPMPS_ERR_STATE = 8,            /* call out of order (e.g. no Hamiltonian or MPS set)  */
    SPMPS_ERR_UNSUPPORTED = 9       /* valid request the library does not implement       */
} spmps_status;

typedef struct {
    int batched;        /* 1: one grouped launch per contraction phase over all beta points and
                           blocks (default); 0: one launch per beta point and phase          */
    int precond;        /* Davidson correction: 0 = diagonal (default), 1 = metric CG,
                           2 = learned (spmps_mlp_*; the diagonal correction replaces it for the
                           rest of a solve once |r| has not improved by 10 % in 12 iterations,
                           and when its direction lies in the basis),
                           3 = Olsen: the diagonal correction plus eps M^-1 N x with eps making
                           it N-orthogonal to x (M = diag H - theta diag N),
                           4 = metric blocks: t = (N_eff + s I)^-1 r with s = 1e-7.  N_eff is the
                           network of the rotated identity MPO (Fig. spmpsOpt (c)); every factor
                           conserves the particle number of its part, so N_eff is exactly
                           block-diagonal in (N of the left bond index, n(s1), n(s2)).  The blocks
                           are assembled densely and factorised (FP64 Cholesky) once per two-site
                           step.  The converged x, defined modulo ker N_eff, is replaced by the
                           representative (N_eff + s I)^-1 N_eff x before decimation.  Blocks above
                           metric_max_dim keep the diagonal correction (and x there); all of them
                           do when the factors would exceed 8 GB or a pivot is not positive. */
    int cg_steps;       /* CG steps on N_eff t = r for precond == 1 (default 5)               */
    double dav_tol_r;   /* Davidson residual norm tolerance (default 1e-6)                    */
    double dav_tol_theta; /* Davidson eigenvalue change tolerance (default 1e-10)             */
    int dav_max_sub;    /* Davidson subspace size before restart (default 20, max 32)         */
    int dav_max_iter;   /* Davidson iteration cap per two-site step (default 200)             */
    int device;         /* CUDA device ordinal (default 0)                                    */
    int jacobi_smem_max; /* decimation blocks handled by one CTA (dimension <= 64 or > 256) up to
                            this size are diagonalised in shared memory, larger ones in global
                            memory (default and maximum 112; 0 = default); blocks of dimension
                            65..256 always run on an 8-CTA thread-block cluster */
    int precision;      /* bulk H_eff x block products: 0 = FP64 (default), 1 = TF32, 2 = 3xTF32
                           (tensor cores, FP32 accumulation).  N_eff x, environments, Davidson and
                           decimation stay FP64; with 1 or 2 each Davidson solve starts with
                           reduced-precision actions (keeping only subspace directions whose
                           N-norm is well above the precision of the products) and switches to
                           FP64 actions in the same subspace once |r| < max(1e-5, 1e-6 |theta|)
                           (3xTF32) or max(1e-3, 1e-3 |theta|) (TF32; also when |r| stagnates), at
                           the latest at half of dav_max_iter, then converges to the FP64
                           tolerance. */
    int autotune;       /* 1: the first projected-action plan of each site times the candidate
                           tile policies of the block GEMMs (phases A and C separately, CUDA
                           events, a few actions on scratch vectors) and keeps the fastest for
                           that site; 0 (default): the fixed least-padding policy. */
    int metric_max_dim; /* precond == 4: largest metric block that is factorised (0 = default 3072) */
    int tc_wait_polls;  /* polls of the bounded mbarrier wait for the tensor-core MMAs of the learned
                           correction before it gives up with SPMPS_ERR_TIMEOUT (0 = default 2^24,
                           about a second); after giving up the kernel still waits, with the default
                           limit, for its MMAs in flight and frees its tensor memory; the same
                           limit applies to the stacked tcgen05 GEMM of the H products and to the
                           split-product GEMM (fp64_tensor_cores), whose give-ups the next Davidson
                           iteration reports as SPMPS_ERR_TIMEOUT (and clears); spmps_apply_heff
                           does not read their status word */
    int tensor_core_kernel; /* precision 1 or 2: 0 = the stacked tcgen05 GEMM (kind::tf32, operands
                           staged in shared memory, accumulator in tensor memory; tasks sharing
                           their B operand stacked along M) (default), 1 = the warp-level
                           mma.sync.m16n8k8 kernel on the same task lists */
    double m_screen;    /* approximate M-sector screening (Sec. 2.3.1, closing paragraph), 0 = off
                           (default): per operator, beta point and MPO channel, the block products
                           whose environment sub-block between a bra label and a ket label (M mixed
                           by the rotation) has a Frobenius norm below m_screen times the largest
                           such sub-block of the channel are dropped from phases A and C.  An
                           approximation: y and z change by amounts of the order of m_screen;
                           spmps_apply_flops reports the reduced work. */
    int fp64_tensor_cores; /* 1: the FP64 block products of phases A and C of every projected action
                           (H and N, both whenever they are computed in FP64) run on the tensor
                           cores as exact products of 8-bit digits: per K stage of 32, each entry
                           is cut into seven signed base-256 digits against the exponent of its row
                           (A) or column (B) maximum, the digit products of each level p + q = 2..9
                           are summed exactly in an FP32 tensor-memory accumulator by
                           tcgen05.mma kind::f16 (every partial sum an integer below 2^24), and the
                           levels are combined in FP64 (the splitting scheme of Ozaki, Ogita, Oishi
                           and Rump, Numer. Algorithms 59, 2012).  The error per stage is of the
                           order of 32 * 2^-55 max|a_i.| max|b_.j|, the size of FP64 rounding;
                           0 (default): the FP64 pipe. */
} spmps_options;

/* Fill *opt with the defaults listed above. */
void spmps_default_options(spmps_options* opt);

/* Create a handle for K spatial orbitals, N electrons, spin projection M = twoM/2, target spin
 * S = twoS/2, n_beta Gauss-Legendre points (Eq. pmpo) and maximal bond dimension D.
 * Checks (SPMPS_ERR_BAD_INPUT): K >= 2, D >= 1, n_beta >= 1, 0 <= N <= 2K, N + twoM even,
 * twoS >= |twoM|, twoS + N even, both electron counts in [0, K].  n_beta below the exactness
 * bound of Eq. exactQuadrature is accepted (the projector is then approximate).
 * opt may be NULL (defaults).  On success *out receives the handle. */
spmps_status spmps_create(int K, int N, int twoM, int twoS, int n_beta, int D,
                          const spmps_options* opt, spmps_handle* out);

spmps_status spmps_destroy(spmps_handle h);

/* Last error message of the handle (static storage when h is NULL); never NULL. */
const char* spmps_last_error(spmps_handle h);

/* Hamiltonian of an open Hubbard chain over the K sites (Sec. 4.1 with a 1D lattice):
 * H = -t sum_{k,s} (a+_{k s} a_{k+1 s} + h.c.) + U sum_k n_{k alpha} n_{k beta}. */
spmps_status spmps_set_hubbard(spmps_handle h, double t, double U);

/* General Hamiltonian of Eq. sqH from one-electron integrals h1 (K*K, row-major) and
 * chemist two-electron integrals h2 = (pq|rs) (K^4 row-major, may be NULL) plus e_core
 * (Eq. sumH: the paper's g_{pq,sr} = <pq|sr> = (ps|qr)).  Inputs are copied.  h1 must be
 * symmetric and h2 Hermitian ((pq|rs) = (qp|sr)), else SPMPS_ERR_BAD_INPUT.  Integrals that
 * couple only nearest neighbours (h1) and single orbitals ((pp|pp)) get the bond-dimension-6
 * Hubbard-like MPO; all others the general MPO (Eq. sumH / Eq. Wfac): every term placed with
 * complementary-operator channels, bond dimension 2 + 2 n_L + 2 n_R + O(min(n_L, n_R)^2) at a
 * cut with n_L / n_R spin-orbitals on its sides.  The MPO site tensors live on the host (one
 * copy per beta point); when they would need more than 4 GB the call returns
 * SPMPS_ERR_UNSUPPORTED. */
spmps_status spmps_set_hamiltonian(spmps_handle h, const double* h1, const double* h2, double ecore);

/* Hamiltonian given directly as an MPO on spatial sites (an alternative to the integrals):
 * bond_dims[0..K] (bond_dims[0] = bond_dims[K] = 1) and sites[k] = W[k] as a dense row-major
 * (bond_dims[k], bond_dims[k+1], 4, 4) array, W[wl][wr][s][t] = <s| op |t> in the local basis
 * {0, b, a, ab} (index 2 n_alpha + n_beta) with the Jordan-Wigner order of Eq. JWtrans.  The
 * operator must conserve the particle number (checked: SPMPS_ERR_BAD_INPUT) and be Hermitian
 * (not checked).  Inputs are copied. */
spmps_status spmps_set_mpo(spmps_handle h, const int* bond_dims, const double* const* sites);

/* Host-only (no device, no handle): the general MPO the library builds from integrals (same
 * conventions as spmps_set_hamiltonian and spmps_set_mpo, without the Hermiticity check).
 * First call with sites == NULL fills bond_dims[0..K]; the second copies W[k] into sites[k]
 * (bond_dims[k] * bond_dims[k+1] * 16 doubles each). */
spmps_status spmps_mpo_from_integrals(int K, const double* h1, const double* h2, double ecore, int* bond_dims,
                                      double* const* sites);

/* Initial MPS: the product state of a Slater determinant (Eq. FSMPS
 * with all bond dimensions 1): occ[k] in {0 = empty, 1 = beta, 2 = alpha, 3 = both} for each
 * spatial orbital k (the local index 2 n_alpha + n_beta).  The occupations must give the
 * handle's (N, 2M), else SPMPS_ERR_BAD_INPUT.  Bond dimensions grow up to D in the two-site
 * sweeps.  The centre is site 0. */
spmps_status spmps_init_determinant(spmps_handle h, const int8_t* occ);

/* Random initial MPS with the handle's (N, 2M) and bond dimension D: on every bond the labels
 * (n, 2m) reachable from the left and completable on the right, dimensions in proportion to the
 * smaller of the left and right Fock-sector sizes (largest-remainder rounding, total <= D),
 * labels without a live neighbour removed; entries i.i.d. N(0, 1) from a SplitMix64 counter
 * stream (Box-Muller) of `seed`; then canonicalised (spmps_canonicalize). */
spmps_status spmps_init_random(spmps_handle h, uint64_t seed);

/* Checkpoint file of the current MPS (labels, site tensors, centre, and the problem's K, N,
 * 2M, 2S) in a little-endian binary format: 8-byte magic "SPMPSCK1", six int32 (K, N, 2M, 2S,
 * centre, 0), the K+1 bond dimensions (int32), 2 int32 labels (n, 2m) per bond index, then the
 * site tensors (D_k, 4, D_k+1) as float64.  spmps_load reads it into a handle with the same
 * K, N and 2M (else SPMPS_ERR_BAD_INPUT) through spmps_set_mps. */
spmps_status spmps_save(spmps_handle h, const char* path);
spmps_status spmps_load(spmps_handle h, const char* path);

/* Load an MPS.  bond_dims[i] (i = 0..K) is the dimension of bond i (bond_dims[0] =
 * bond_dims[K] = 1); labels holds 2*sum(bond_dims) ints: (n, 2m) per bond index, bond by bond,
 * sorted as described above; sites[k] points to a dense row-major D_k x 4 x D_{k+1} array
 * (entries outside the (N, M) pattern are ignored).  The orthogonality centre is declared
 * by `center`: sites left of it must be left-canonical and sites right of it right-canonical
 * for energies to be meaningful (the contractions themselves do not need it). */
spmps_status spmps_set_mps(spmps_handle h, const int* bond_dims, const int* labels,
                           const double* const* sites, int center);

/* Number of entries of the two-site tensor at sites (site, site+1) and its block table:
 * for block j (j < *n_blocks) blocks[5j .. 5j+4] = (index of the left label in bond `site`,
 * s = 4*s1 + s2, offset of the block's first column inside its row block, rows, columns);
 * row_block_offsets[i] / row_block_widths[i] give, per left label i, the offset of its row
 * block and its width W.  Any output pointer may be NULL; array sizes are at most
 * 16 * (labels of bond `site`) for blocks and (labels of bond `site`) for the two others. */
spmps_status spmps_x_layout(spmps_handle h, int site, int64_t* n_x, int* n_blocks, int* blocks,
                            int64_t* row_block_offsets, int* row_block_widths, int* n_left_labels);

/* The projected actions of Eq. geproblem at sites (site, site+1):
 *   y = sum_g c_g Pi_(N,M) [ H exp(-i beta_g S_y) ]_eff x,   z = sum_g c_g Pi_(N,M) [ exp(-i beta_g S_y) ]_eff x
 * (Fig. spmpsOpt (b), (c)) with the environments of the current MPS, built on demand.
 * x, y, z are DEVICE pointers in the row-block layout (n_x doubles each, x read-only; y or z
 * may be NULL to skip that output).  stream is a cudaStream_t (NULL: the handle's stream);
 * the call is asynchronous with respect to the host except when environments must be built.
 * The H part uses the handle's precision option (FP64, TF32 or 3xTF32 block products); z is FP64. */
spmps_status spmps_apply_heff(spmps_handle h, int site, const double* x, double* y, double* z,
                              void* stream);

/* Same action, with CUDA events recorded on `stream` between the phases; phase_ms[0..3]
 * receive the durations of the zero fill, the environment GEMMs over x (phase A), the MPO-leg
 * combination (phase B) and the output GEMMs (phase C); the call synchronises the stream. */
spmps_status spmps_apply_heff_timed(spmps_handle h, int site, const double* x, double* y, double* z,
                                    void* stream, double* phase_ms);

/* Algorithmic flops of one call of spmps_apply_heff at `site`, split as [A, B, C] (symmetry-
 * allowed block products only: 2*m*n*k per block GEMM, 2*rows*cols per MPO-leg term). */
spmps_status spmps_apply_flops(spmps_handle h, int site, double* flops3);

/* Algorithmic flops and bytes of one call of spmps_apply_heff at `site`, per operator (op 0 = H,
 * 1 = N) and phase (index 3*op + phase, phase 0 = A, 1 = B, 2 = C).  Flops as spmps_apply_flops.
 * Bytes, 8 per element: phase A reads the op's left environment and x and writes T1, each once
 * per beta point; phase B reads T1 and writes T3; phase C reads T3 and the op's right environment
 * and writes the per-beta partial outputs (the HBM roofline numerators).  Either pointer may be
 * NULL (6 doubles each otherwise). */
spmps_status spmps_apply_costs(spmps_handle h, int site, double* flops6, double* bytes6);

/* FP64 fused multiply-add throughput of `device` in TFLOP/s, measured by a kernel of
 * independent FMA chains on every SM (the roofline denominator of the FP64 path). */
spmps_status spmps_device_fp64_peak(int device, double* tflops);

/* Dense TF32 tensor-core throughput of `device` in TFLOP/s (2 flops per multiply-add), measured on
 * `sms` SMs (0 = all), one CTA per SM: kind 0 = the warp-level mma.sync.m16n8k8 TF32 instruction
 * with FP32 accumulation (32 warps, 8 independent chains per warp), kind 1 =
 * tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, operands in shared memory, accumulator in tensor
 * memory, issued by one thread of one CTA per SM; kind 2 = the warp-level INT8 instruction
 * mma.sync.m16n8k32 s8 x s8 -> s32 (tera-operations per second: the rate an integer-split FP64
 * emulation would build on).  The roofline denominators of the reduced-precision action.
 * SPMPS_ERR_TIMEOUT if the bounded wait for the tcgen05 MMAs gave up. */
spmps_status spmps_device_tf32_peak(int device, int kind, int sms, double* tflops);

/* The same projected action as spmps_apply_heff, for callers that cannot let the library allocate
 * device memory when they need it: callers whose device memory is reserved up front by their own
 * pool allocator, or embedding runtimes that forbid the CUDA allocator after start-up.  The paper
 * has no counterpart; this is an interface variant only.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its intermediates live in one
 * file-scope device array of 4 Mi doubles (32 MiB) that every GPU loading the library keeps until
 * exit; problems needing more return SPMPS_ERR_BAD_INPUT.  The H part always runs FP64-accurate (as
 * spmps_apply_heff with precision 0: on the FP64 pipe, or as split products on the tensor cores
 * when fp64_tensor_cores is set), whatever the handle's precision option.  The environments
 * and contraction plan of `site` must already exist (a previous spmps_apply_heff or spmps_energy
 * call for that site builds them, and allocates); otherwise SPMPS_ERR_STATE.  All calls share the
 * array, which keeps the last call's contents (the call zeroes what must start at zero): calls
 * that overlap on the GPU race and must be serialised.  When `stream` is not the handle's stream,
 * the call orders it after the work already queued on the handle's stream (an event; the first
 * such call on a handle creates it).  The first call on each device looks up the array's address
 * (cudaGetSymbolAddress).  The per-launch profiler (spmps_profile) does not record this call.
 * Arguments as in spmps_apply_heff. */
spmps_status spmps_apply_heff_noalloc(spmps_handle h, int site, const double* x, double* y, double* z,
                                      void* stream);

/* Same action with HOST buffers: copies x to the device, applies, copies y and z back
 * (synchronous). */
spmps_status spmps_apply_heff_host(spmps_handle h, int site, const double* x, double* y, double* z);

/* The current two-site tensor A[site] A[site+1] into a DEVICE buffer of n_x doubles. */
spmps_status spmps_two_site(spmps_handle h, int site, double* x);

/* Canonicalise the loaded MPS on the device: right-canonical sites 1..K-1, centre on site 0,
 * norm 1.  Labels whose rank is zero are removed (bond dimensions may shrink). */
spmps_status spmps_canonicalize(spmps_handle h);

/* n_sweeps two-site sweeps (left-to-right steps k = 0..K-3, then right-to-left k = K-2..0;
 * centre must be on site 0).  Per step: generalised Davidson for H_eff x = theta N_eff x,
 * SVD decimation to D (Sec. 2.3.1), environment update.  energies[s] (may be NULL) receives the
 * energy after sweep s.  Returns SPMPS_ERR_NOT_CONVERGED if any Davidson hit its cap (the
 * sweep still completes). */
spmps_status spmps_sweep(spmps_handle h, int n_sweeps, double* energies);

/* One two-site step at sites (site, site+1) with the centre inside the pair: generalised
 * Davidson from the current two-site tensor, decimation to D, environment update.
 * move_right != 0 leaves site `site` left-canonical and the centre on site+1; otherwise site+1
 * becomes right-canonical and the centre moves to `site`.  theta (may be NULL) receives the
 * lowest generalised eigenvalue, iterations (may be NULL) the Davidson iteration count.
 * Returns SPMPS_ERR_NOT_CONVERGED (after finishing the step) when Davidson hit its cap. */
spmps_status spmps_optimize_step(spmps_handle h, int site, int move_right, double* theta, int* iterations);

/* Energy functional (Eq. efunctional) and <Psi|P|Psi> at the current centre. */
spmps_status spmps_energy(spmps_handle h, double* E, double* norm_P);

/* <S^2> of the projected state, through the same engine with the S^2 MPO of Eq. Sfac. */
spmps_status spmps_expect_s2(spmps_handle h, double* s2);

/* Spin-free properties (Eq. PropSpinFree): <O> = <Psi|O P|Psi> / <Psi|P|Psi> for an operator
 * that commutes with the projector, through the same environments and projected action as the
 * energy.  Each call builds the environments of O for every beta point (the handle's own
 * environments are kept).  Errors as spmps_energy.
 *
 * spmps_expect_mpo: O given as an MPO in the spmps_set_mpo format (inputs copied).
 * spmps_fragment_energies: e[p] (p = 0..K-1), the terms of Eq. sumH whose first creation operator
 *   is on spatial orbital p, both spins: sum_p e[p] + e_core = E.  Needs the integrals of
 *   spmps_set_hamiltonian or spmps_set_hubbard (SPMPS_ERR_STATE after spmps_set_mpo).
 * spmps_rdm1: the spin-free one-particle density matrix gamma[p*K + q] = <E_pq>,
 *   E_pq = sum_s a+_ps a_qs (K*K doubles; symmetric for the real wavefunctions of this library).
 * spmps_spin_correlation: <S_X . S_Y> for orbital sets X (nx indices) and Y (ny indices).
 * spmps_seniority: <Omega>, the number of singly occupied orbitals. */
spmps_status spmps_expect_mpo(spmps_handle h, const int* bond_dims, const double* const* sites, double* value);
spmps_status spmps_fragment_energies(spmps_handle h, double* e);
spmps_status spmps_rdm1(spmps_handle h, double* gamma);
spmps_status spmps_spin_correlation(spmps_handle h, const int* X, int nx, const int* Y, int ny, double* value);
spmps_status spmps_seniority(spmps_handle h, double* value);

/* Statistics: counts[0] = Davidson iterations of the last sweep, counts[1] = projected applies
 * issued, counts[2] = kernel launches issued by the library since the handle was created;
 * values[0] = algorithmic flops of one projected apply at the last site applied (symmetry-
 * allowed block products only), values[1] = discarded weight of the last sweep, values[2] =
 * algorithmic flops of every projected apply issued since the handle was created.  Either
 * pointer may be NULL (counts holds 3, values 3). */
spmps_status spmps_stats(spmps_handle h, int64_t* counts, double* values);

/* Davidson iterations of the last spmps_sweep call: *iterations counts every iteration, and
 * *refine_iterations those after the switch from the TF32 / 3xTF32 action to the FP64 action
 * (0 with precision 0).  Both are reset when spmps_sweep starts.  Either pointer may be NULL. */
spmps_status spmps_davidson_stats(spmps_handle h, int64_t* iterations, int64_t* refine_iterations);

/* Copy the current MPS to host memory (checkpoint).  First call with sites == NULL: fills
 * bond_dims[0..K] (and *center).  Second call: labels must hold 2 * sum(bond_dims) ints and sites[k]
 * D_k * 4 * D_{k+1} doubles (dense row-major, zeros outside the (N, M) pattern) -- the format
 * spmps_set_mps reads.  Any pointer other than bond_dims may be NULL. */
spmps_status spmps_get_mps(spmps_handle h, int* bond_dims, int* labels, double* const* sites, int* center);

/* The cudaStream_t the handle's own work (sweeps, environment builds) runs on. */
spmps_status spmps_stream(spmps_handle h, void** stream);

/* Per-launch CUDA-event timing of the library's block-GEMM and MPO-leg kernels (off by default).
 * enable != 0 switches it on and clears the counters; enable == 0 switches it off. */
spmps_status spmps_profile(spmps_handle h, int enable);

/* Counters of the profiler for `kind`: 0 = k_gemm_f64 launches, 1 = k_comb_f64 launches (their
 * algorithmic flops, same rule as spmps_apply_flops), 2 = the Davidson Ritz step (k_ritz),
 * 3 = the rest of each Davidson iteration outside the projected action (dots, gemv, residual,
 * Gram-Schmidt), 4 = the decimation eigen-solve and truncation, 5 = host time spent building and
 * uploading contraction plans (ms of host clock, launches = plans built), 6 = assembly and
 * factorisation of the metric blocks (precond 4, once per two-site step), 7 = the per-iteration
 * solves with them, 8 = the reduced-precision block-GEMM launches (TF32 / 3xTF32 H products;
 * kind 0 then counts the FP64 ones only), 9 = the FP64-accurate split-product GEMM launches
 * (fp64_tensor_cores; kind 0 then counts only the block products outside projected actions).
 * Synchronises the handle's stream. */
spmps_status spmps_kernel_stats(spmps_handle h, int kind, int64_t* launches, double* ms, double* flops);

/* ---- Learned Davidson correction (no counterpart in the paper) ------------------------------
 * A perceptron 4 -> 256 -> 256 -> 1 (ReLU) maps, per element i of the two-site vector, the features
 *   ( sqrt(n) r_i/|r|, sqrt(n) d_i/|d|, dn_i, tanh((dh_i - theta dn_i)/(1+|theta|)) ),
 *   d = -r / (dh - theta dn) clamped to |.| >= 1e-4 (the diagonal correction),
 * to a correction t_i; dh, dn are the diagonals of H_eff and N_eff, r the residual.  Parameters
 * are one float vector: W1 (4 x 256 row-major), b1 (256), W2 (256 x 256 row-major [in][out]),
 * b2 (256), w3 (256), b3 (1): 67329 floats.  With precond = 2 the correction is evaluated with the
 * 256 x 256 layer on the tensor cores (BF16 operands, FP32 accumulation). */

/* Harvest training pairs during Davidson solves (any preconditioner): for each of the first 32
 * iterations of a solve, features at samples_per_iteration evenly spaced elements, with the
 * target sqrt(n) e_i/|e|, e = x* - alpha x_j the part of the converged vector x* not along the
 * current Ritz vector x_j.  capacity = total pairs kept on the device; when enabling with a
 * larger capacity the buffer grows and earlier pairs are cleared; disabling keeps the pairs. */
spmps_status spmps_mlp_harvest(spmps_handle h, int enable, int samples_per_iteration, int64_t capacity);

/* Number of harvested pairs; features (4 per pair) and targets (may be NULL) copied to the host. */
spmps_status spmps_mlp_data(spmps_handle h, int64_t* count, float* features, float* targets);

/* set != 0: load 67329 parameters from the host (layout above); set == 0: read them back. */
spmps_status spmps_mlp_params(spmps_handle h, float* params, int set);

/* Mean squared error of the network on a host batch (X: B x 4, T: B) and its gradients with
 * respect to every parameter (FP32 forward and backward on the device). */
spmps_status spmps_mlp_loss_grad(spmps_handle h, const float* X, const float* T, int B, double* loss, float* grads);

/* `steps` Adam steps (lr, beta1 0.9, beta2 0.999) on minibatches of `batch` harvested pairs drawn
 * with SplitMix64(seed, step, position); reinit != 0 (or no parameters yet) starts from He-normal
 * weights drawn from the same generator.  Returns the first and last minibatch loss. */
spmps_status spmps_mlp_train(spmps_handle h, int steps, int batch, double lr, uint64_t seed, int reinit,
                             double* loss_first, double* loss_last);

/* The network's correction for host vectors r, dh, dn (n each) and theta; tensor_cores != 0
 * runs the BF16 tensor-core path used inside Davidson, 0 an FP32 reference path. */
spmps_status spmps_mlp_infer(spmps_handle h, const double* r, const double* dh, const double* dn, double theta,
                             int64_t n, double* t, int tensor_cores);

/* ---- State-specific excited states (Sec. 2.3.2, Eq. orthoB, Fig. spmpsex) ---------------------
 * spmps_add_lower_state: a lower state |Psi_j> (an MPS with the handle's K, N and 2M, format of
 *   spmps_set_mps; copied; at most 16).  From then on every two-site step (spmps_sweep,
 *   spmps_optimize_step) builds B_j = <Psi_j| P |d Psi / d x> at its sites from per-beta
 *   environments between the running state (bra) and |Psi_j> (ket), orthonormalises the B_j (QR by
 *   Gram-Schmidt twice) into V and solves Eq. geproblem in the range of Q = 1 - V V^T: the start
 *   vector, the residual and every new Davidson direction are projected with Q, so the optimised
 *   state keeps <Psi_j|P|Psi> = 0.  Adding a lower state invalidates the handle's environments.
 * spmps_clear_lower_states: back to the ground-state problem.
 * spmps_lower_overlap: <Psi_j| P |Psi> of the current MPS (B_j . x at the centre pair). */
spmps_status spmps_add_lower_state(spmps_handle h, const int* bond_dims, const int* labels, const double* const* sites);
spmps_status spmps_clear_lower_states(spmps_handle h);
spmps_status spmps_lower_overlap(spmps_handle h, int j, double* value);

/* Quadrature used by the handle: beta_g and c_g (n_beta each, host arrays). */
spmps_status spmps_quadrature(spmps_handle h, double* beta, double* c);

#ifdef __cplusplus
}
#endif
#endif /* SPMPS_H */
