/*
 * lbm_mrt.h -- C ABI of the GB300 (sm_103a) MRT lattice Boltzmann library.
 *
 * The library implements the rectangular multiple-relaxation-time lattice Boltzmann method of
 * Shi, Yuan & Chai, "A unified MRT-LB framework for Navier-Stokes and nonlinear
 * convection-diffusion equations and beyond" (arXiv 2512.16230): the two-level full-correction
 * scheme Eq. (2-3) with the Hermite-moment collision Eq. (H-MRT-LB-1) on the multispeed
 * rectangular lattices of Sec. 5 and App. C/D (rD2Q25/21/17/13, rD3Q53/45/33).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Lattice units: dt = 1, dx_1 = 1, c_a = dx_a / dx_1 (Sec. 5, "c_alpha = dx_alpha / dt").
 *  - A grid has n[0] x n[1] (x n[2]) cells, periodic in every direction. Every field is a
 *    dense C-order array with x fastest: element (x, y, z) sits at ((z * n[1]) + y) * n[0] + x.
 *    Vector fields are structure-of-arrays: u[a * ncells + cell]. Populations are
 *    f[i * ncells + cell] with i in the paper's velocity order.
 *  - Host/device: arguments named *_host live in host memory; arguments accompanied by an
 *    `on_device` flag live in device memory of the model's GPU when the flag is non-zero and in
 *    host memory otherwise. Field and population I/O is always FP64.
 *  - Ownership: the caller owns every buffer it passes. The library owns the handles and, unless
 *    the caller supplies a workspace, the device memory of a model. Nothing is retained past the
 *    call except handles and workspaces.
 *  - Streams: a model runs all its kernels on the CUDA stream given at creation (NULL = the
 *    legacy default stream). lbm_model_step and lbm_model_stream_only are asynchronous; the
 *    calls that return data to host memory synchronize the stream first.
 *  - Errors: every call returns an lbm_status and never throws; on failure lbm_last_error()
 *    returns a thread-local message. A failed call leaves the model as it was before the call
 *    except where stated. No call faults the GPU on bad arguments: sizes and pointers are
 *    validated on the host first.
 *  - FP64 runs only in the lattice set-up (lbm_lattice_create) and in the conservation sums;
 *    the time step computes in the model's compute dtype.
 */
#ifndef LBM_MRT_H
#define LBM_MRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 1

typedef struct lbm_lattice lbm_lattice; /* opaque, library-owned */
typedef struct lbm_model lbm_model;     /* opaque, library-owned */
typedef struct lbm_batch lbm_batch;     /* opaque, library-owned */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,                /* invalid argument (null pointer, size, axis, dtype mix) */
  LBM_ERR_LATTICE_INFEASIBLE = 2, /* a Hermite norm N_r <= 0 or HWH^T not diagonal */
  LBM_ERR_OOM = 3,                /* device allocation failed or workspace too small */
  LBM_ERR_CUDA = 4,               /* a CUDA runtime call failed (message has the CUDA error) */
  LBM_ERR_NONFINITE = 5,          /* a conservation sum is NaN or infinite */
  LBM_ERR_NOT_IMPLEMENTED = 6,
  LBM_ERR_TIMEOUT = 7             /* a device-side bounded wait ran out (reported by syncing calls) */
} lbm_status;

/* Lattices of Sec. 5 and App. D, velocity columns in the paper's printed order. */
typedef enum {
  LBM_RD2Q13 = 0, /* Eq. (Q13lattice)                                    */
  LBM_RD2Q17 = 1, /* Eq. (3-1) with w21 = w17 = w18 = 0 (Sec. 5 (ii))    */
  LBM_RD2Q21 = 2, /* Eq. (3-1) with w21 = 0 (Sec. 5 (i))                 */
  LBM_RD2Q25 = 3, /* Eq. (3-1)                                           */
  LBM_RD3Q33 = 4, /* App. D, rD3Q33                                      */
  LBM_RD3Q45 = 5, /* App. D, rD3Q53 with w45 = 0 (the eight (+-2)^3 vectors dropped) */
  LBM_RD3Q53 = 6, /* App. D, rD3Q53                                      */
  LBM_RD2Q9 = 7,  /* single-speed rectangular D2Q9 (Sec. 3.4, k = 1): rD2Q25's first 9 columns */
  LBM_RD3Q27 = 8  /* single-speed rectangular D3Q27 (k = 1): rD3Q53's first 27 columns       */
} lbm_kind;

typedef enum {
  LBM_F64 = 0,     /* IEEE binary64 */
  LBM_F32 = 1,     /* IEEE binary32 */
  LBM_BF16_DEV = 2, /* storage only: bfloat16 deviation f_i - w_i * rho_ref */
  LBM_F16_DEV = 3  /* storage only: binary16 deviation f_i - w_i * rho_ref */
} lbm_dtype;

typedef enum {
  LBM_NSE = 0, /* isothermal Navier-Stokes, Sec. 3 with the multispeed choices of Sec. 3.4 */
  LBM_NCDE = 1 /* nonlinear convection-diffusion, App. A */
} lbm_eq;

typedef enum {
  LBM_NCDE_MOMENT = 0, /* nonlinearity in M2 = cs2_eq D(phi) I, constant S1 (default)          */
  LBM_NCDE_RATE = 1,   /* D(phi) = phi, per-cell S1(phi) giving K(phi) = K0 (1 + nonlin phi^2) */
  LBM_NCDE_CDE = 2     /* diffusion-based CDE, App. A special case (3)                        */
} lbm_ncde_variant;

/* How the CUDA-core collide-stream kernel of 16-bit storage gathers the pull sources. */
typedef enum {
  LBM_GATHER_AUTO = 0,    /* rows when they apply (default), threads otherwise                 */
  LBM_GATHER_THREADS = 1, /* every thread loads its Q sources from global memory               */
  LBM_GATHER_ROWS = 2     /* bulk copies of whole source x-rows into shared memory             */
} lbm_gather;

int lbm_abi_version(void);

/* Thread-local description of the last error returned on this thread ("" if none). */
const char* lbm_last_error(void);

/* ------------------------------------------------------------------------------------------
 * Lattices
 * ------------------------------------------------------------------------------------------ */

/* Build lattice `kind` on the current CUDA device, in FP64, on the GPU:
 *   - weights from the printed closed forms: Eq. (WeightQ25) (rD2Q25 and its sub-lattices),
 *     Eq. (Q13lattice), the rD3Q53 and rD3Q33 weight lists of App. D, with
 *     d_0a = cs2[a] / c[a]^2 (the definition stated with Eq. (new11)); the single-speed rD2Q9 and
 *     rD3Q27 meet only sum w = 1, Delta2_aa = cs2[a] and the mixed fourth/sixth moments (their
 *     axis fourth moment is c_a^2 cs2[a], the delta^(4) anisotropy of k = 1), which gives the
 *     product of the 1D weights 1 - d_0a and d_0a / 2;
 *   - Hermite rows H0..H3 (Sec. 5) by weighted Gram-Schmidt of the monomials in the paper's row
 *     order, which yields the rectangular-cell correction of the third-order rows of
 *     Eq. (CorrectQ25) and App. D; on the single-speed lattices the pure cubes c_a^3 equal
 *     c_a^2 c_a and are left out (R = 8 in 2D, 17 in 3D; 10 and 20 otherwise), and their
 *     equilibrium takes M30 = 0, the standard-lattice case of Sec. 3.4;
 *   - norms N_r = sum_i w_i H_ri^2 and a check that H W H^T is diagonal.
 * c[d]      axis speeds c_a = dx_a / dx_1 (c[0] = 1 in lattice units), host memory.
 * cs2[d]    squared sound speed per axis c_sa^2 (Remark 2; equal values = isotropic), host.
 * free_w    the free weights, host memory (may be NULL when n_free == 0), in this order:
 *             rD2Q25: w13, w17, w18, w21     rD2Q21: w13, w17, w18     rD2Q17: w13
 *             rD3Q53: w45                    rD2Q13, rD3Q45, rD3Q33, rD2Q9, rD3Q27: none
 * Negative weights are allowed (reported by lbm_lattice_query). Synchronous.
 * Errors: LBM_ERR_ARG (bad kind, n_free, c <= 0, cs2 <= 0), LBM_ERR_LATTICE_INFEASIBLE,
 *         LBM_ERR_CUDA. On success *out receives a new handle. */
lbm_status lbm_lattice_create(lbm_kind kind, const double* c, const double* cs2,
                              const double* free_w, int n_free, lbm_lattice** out);

/* Copy the lattice tables to host memory. Every output pointer may be NULL.
 *   d, Q, R : dimension, number of velocities, number of Hermite rows of order <= 3
 *   e[Q*d]  : integer velocity components (c_i = diag(c) e_i)
 *   w[Q]    : weights;  H[R*Q]: Hermite rows on the lattice (row-major);  N[R]: norms
 *   T[R*R]  : H_r(c) = sum_k T[r*R + k] * mono_k(c), mono_k the monomials in the paper's row
 *             order (2D: 1,x,y,xx,xy,yy,xyy,xxy,xxx,yyy; 3D: App. D, M1..M20). */
lbm_status lbm_lattice_query(const lbm_lattice* lat, int* d, int* Q, int* R, int8_t* e,
                             double* w, double* H, double* N, double* T);

/* Rows of order >= 4 that complete the Q x Q Hermite matrix (the paper leaves them to the
 * designer, Sec. 5 / App. D): monomials of degree 4, 5, ... kept in graded order when they raise
 * the rank, each W-orthogonalised against every earlier row, so that the rows of order k span
 * the W-orthogonal complement of the orders < k within the lattice functions of degree <= k.
 * Built in FP64 by lbm_lattice_create. Every output pointer may be NULL.
 *   n_high        Q - R;   orders[n_high]: the order of each row (even orders first, then odd)
 *   H[n_high*Q]   the rows on the lattice (row-major, each scaled to unit max);  N[n_high]: W-norms
 * Errors: LBM_ERR_ARG (NULL lattice), LBM_ERR_LATTICE_INFEASIBLE (a row has zero W-norm because
 *         some weights are zero, or the monomials do not reach rank Q). */
lbm_status lbm_lattice_query_high(const lbm_lattice* lat, int* n_high, int* orders, double* H,
                                  double* N);

lbm_status lbm_lattice_destroy(lbm_lattice* lat);

/* ------------------------------------------------------------------------------------------
 * Models: one periodic solve on one lattice
 * ------------------------------------------------------------------------------------------ */

/* Device bytes a model needs: two population buffers (Q * ncells * sizeof(store)), the NCDE
 * previous-step field and cross-diffusion field psi (or, for the NSE on rD2Q9 / rD3Q27, two
 * previous-step density fields), the body-force profile and the reduction scratch, each 256-byte
 * aligned. */
lbm_status lbm_model_workspace_bytes(const lbm_lattice* lat, lbm_eq eq, const int64_t* n,
                                     lbm_dtype store, size_t* bytes);

/* Create a model on grid n[d] (host memory). Every n[a] must be at least the largest velocity
 * component of the lattice (2 or 3) and the cell count at most 2^31 - 2^21 = 2,145,386,496 (cell
 * indices are 32-bit in the kernels; the margin keeps every index a launch forms below 2^31).
 * lbm_model_workspace_bytes applies the same checks (LBM_ERR_ARG) without allocating anything.
 * store/compute: (F64, F64), (F32, F32), (BF16_DEV or F16_DEV, F32).
 * stream    : cudaStream_t on which every kernel of the model runs (NULL: legacy default).
 * workspace : device buffer of at least lbm_model_workspace_bytes(), 256-byte aligned, owned by
 *             the caller and kept alive until lbm_model_destroy; NULL lets the library allocate.
 * Defaults: every rate 1 (s_r = s_high = 1), cs2_eq = cs2[0], no body force, u_const = 0,
 * nonlin = 0, populations zero. The model keeps a reference to `lat`, which must outlive it. */
lbm_status lbm_model_create(const lbm_lattice* lat, lbm_eq eq, const int64_t* n, lbm_dtype store,
                            lbm_dtype compute, void* stream, void* workspace,
                            size_t workspace_bytes, lbm_model** out);

/* Diagonal relaxation matrix S in the Hermite basis (Sec. 4, Eq. (H-MRT-LB-1)):
 * s[R] the rate of each Hermite row in the paper's order, s_high the one rate shared by every
 * row of order >= 4. Rates must lie in (0, 2]. The kinematic viscosity of the NSE is
 * nu = cs2_eq (1/s_2 - 1/2) (Eq. (4-29), compressible, k = 0); on the single-speed lattices
 * (k = 1) the normal row c_a^2 - c_sa^2 gives the normal viscosity (1/s_a - 1/2)(c_a^2 - cs2_eq),
 * so s_a = 1 / (2 nu / (c_a^2 - cs2_eq) + 1/2) per axis makes it isotropic. The NCDE
 * diffusivity is K = cs2_eq (1/s_1 - 1/2) (Eq. (ME-NCDE-3)). */
lbm_status lbm_model_set_relaxation(lbm_model* m, const double* s, double s_high);

/* Independent bulk viscosity (NSE): the normal second-order moments relax with the inverse of
 * S2^(1) = diag(1/s_sa) + a b^T / d (Eq. (4-27)), where s_sa are the rates set for the normal rows
 * c_a^2 - c_sa^2. Multispeed lattices (k = 0): a_a = 1/s_bulk - 1/s_sa, b = 1, so that
 * mu = (1/s_s - 1/2) p dt and mu_b = (2/d)(1/s_bulk - 1/2) p dt (Eq. (4-29)). Single-speed
 * lattices (k = 1): a_a = (1/s_bulk - 1/s_sa)(c_a^2 - cs2_eq), b_b = 1/(c_b^2 - cs2_eq) as printed,
 * so that a longitudinal wave along a sees (c_a^2 - cs2_eq)((1/s_sa - 1/2) + (1/s_bulk - 1/s_sa)/d).
 * The same block enters (I - S2/2) M2G. s_bulk <= 0 restores the diagonal relaxation.
 * Errors: LBM_ERR_ARG. */
lbm_status lbm_model_set_bulk(lbm_model* m, double s_bulk);

/* Rates of the rows of order >= 4, one per order (Eq. (H-MRT-LB) with the full Q x Q Hermite
 * matrix; the higher rows as in lbm_lattice_query_high): s_order[k] is the rate of order 4 + k,
 * k < n_orders <= 9; the orders not given relax with s_high. Rates must lie in (0, 2]. Since the
 * equilibrium and the sources have no moments of order >= 4, the update adds
 * -w_i sum_r (s_r - s_high) H_r(c_i) (sum_j H_r(c_j) f_j) / N_r over those rows, which costs the
 * step two more contractions with them. n_orders = 0 restores the shared rate.
 * Inside a batch the solve joins a group of solves with per-order rates (CUDA cores).
 * Errors: LBM_ERR_ARG, LBM_ERR_LATTICE_INFEASIBLE (lattice without complete higher rows). */
lbm_status lbm_model_set_high_rates(lbm_model* m, const double* s_order, int n_orders);

/* Tensor-core (tcgen05) collision. For 16-bit deviation storage (BF16_DEV / F16_DEV) the two contractions
 * of the Hermite-moment collision (Eq. (H-MRT-LB-1)) run as tcgen05 matrix products over tiles
 * of 128 cells with the integer monomial table mono_k(e_i) as the other operand (exact in 16 bits);
 * the per-cell moment-space arithmetic stays in FP32. enable = 0 selects the CUDA-core kernel.
 * With distinct rates for the orders >= 4 (lbm_model_set_high_rates) the higher rows join both
 * products as dense 16-bit operands (the full Q x Q collision). On FP32 storage only the
 * correction of those higher rows runs on the tensor cores, next to the CUDA-core reduced form:
 * it is linear in the pre-collision populations, so it is applied as one dense Q x Q operator
 * G_ij = sum_r a_r H_r(c_i) H_r(c_j) (a_r = -(s_r - s_high) / N_r, built in FP64), one product
 * per 128-cell tile with both operands as FP16 high/low splits of power-of-two scaled values
 * (three products, about 22 bits); without per-order rates FP32 storage always uses the
 * CUDA-core kernel. Default, until this is
 * called: the tensor cores with distinct higher-order rates (there they are the faster kernel),
 * the CUDA cores otherwise.
 * Device-side waits are bounded; a timeout is latched in the model's status word and returned as
 * LBM_ERR_TIMEOUT by the next lbm_model_synchronize / read / get / sums call. After a timeout the
 * populations (and the NCDE / density history fields) are undefined: re-initialise the model
 * (lbm_model_init_fields or lbm_model_set_populations) before stepping it again.
 * enable = 2 is a test hook for that path: the kernel issues no matrix product, every wait runs
 * out after a short limit, the CTAs free their tensor memory and return, and the populations
 * are left undefined.
 * Errors: LBM_ERR_ARG (FP64 storage, enable not in {0, 1, 2}). */
lbm_status lbm_model_set_tensor_cores(lbm_model* m, int enable);

/* Gather of the pull streaming (Eq. (2-2b)) for 16-bit deviation storage on the CUDA cores
 * (the reduced-form collision and lbm_model_stream_only). ROWS: a CTA works on whole x-rows; the
 * source x-row (y - e_y, z - e_z) of each population comes into a shared-memory row buffer by
 * 16-byte asynchronous copies (n_x * 2 bytes per population, counted on an mbarrier, a few rows
 * ahead), every thread reads its sources there at (x - e_x) mod n_x, writes its collided cell
 * back into the buffer, and the row goes to memory by 16-byte stores. It applies when n_x is a
 * multiple of 8 (16-byte rows) and at most 256 cells. THREADS: every thread loads and stores its own cell's
 * populations in global memory. Both give bitwise the same populations.
 * With the tensor cores selected (lbm_model_set_tensor_cores), ROWS runs the two contractions
 * on tcgen05 with the A operands written into tensor memory, also with per-order rates (bitwise
 * the per-thread tcgen05 kernel). AUTO (default) takes ROWS where it applies. Errors: LBM_ERR_ARG
 * for an unknown mode, or ROWS on a model it does not apply to; a step with ROWS forced and
 * per-order rates on the CUDA cores (no row-staged kernel) returns LBM_ERR_NOT_IMPLEMENTED.
 * mode = 3 is a test hook of the bounded waits: ROWS with no row copy issued, so every wait on a
 * row buffer runs out after a short limit, the CTAs return, the next synchronizing call reports
 * LBM_ERR_TIMEOUT and the populations are left undefined. */
lbm_status lbm_model_set_gather(lbm_model* m, lbm_gather mode);

/* Equation of state p = rho * cs2_eq (NSE, Eq. (M-NSEs-6-1)) or the prefactor of the diffusion
 * moment M2 = cs2_eq D(phi) I (NCDE, Eq. (M-NCDE-6)). */
lbm_status lbm_model_set_eos(lbm_model* m, double cs2_eq);

/* NSE body force F(x) = A sin(2 pi k x_b / L_b + phase) e_a, with x_b = i_b c_b the cell
 * coordinate along axis b and L_b = n_b c_b. It enters through M1F = F and the auxiliary moment
 * M2G = (I - S2/2)(uF + Fu) (Eq. (M-NSEs-2), Eq. (M2Ga-1) with S = 0) and the half-force
 * velocity correction of Eq. (2-4-2). A = 0 removes the force. */
lbm_status lbm_model_set_force(lbm_model* m, int axis_a, int axis_b, double A, int k,
                               double phase);

/* NCDE (App. A): constant convection velocity u_const[d] (host) and the nonlinearity of
 * D(phi) = phi + nonlin * phi^3 / 3, i.e. grad D = (1 + nonlin phi^2) grad phi. The auxiliary
 * moment is M1G = (I - S1/2) u (phi^n - phi^{n-1}) (Eq. (M-NCDE-6), M20 = 0). */
lbm_status lbm_model_set_ncde(lbm_model* m, const double* u_const, double nonlin);

/* NCDE variants of App. A (default LBM_NCDE_MOMENT, a1 = 0):
 *   LBM_NCDE_MOMENT  as lbm_model_set_ncde describes;
 *   LBM_NCDE_RATE    M2 = cs2_eq phi I and the first-order rates taken per cell,
 *                    s_a(phi) = 1 / ((1/s_a - 1/2)(1 + nonlin phi^2) + 1/2), so that the
 *                    diffusivity K = cs2_eq (1/s_a(phi) - 1/2) (Eq. (GNCDE-0) read with S1^-1)
 *                    carries the nonlinearity; M1G uses the same per-cell rates;
 *   LBM_NCDE_CDE     the diffusion-based model for d_t phi + u . grad phi = div(K grad phi):
 *                    M1 = 0, M2 = cs2_eq phi I, lambda = 1, S_G = -u . grad phi with the local
 *                    gradient grad_a phi = -s_a M1_a^ne / (dt cs2_eq) (Eq. (M-NCDE-3-00)),
 *                    M0G = (1 - s0/2) S_G (Eq. (M-NCDE-4)), M1G = 0, and phi = sum f + S_G / 2
 *                    (Eq. (2-4-1)); read_fields returns that phi.
 * a1: the mixed-derivative term of Eq. (GNCDE) with A1 = a1 I and B-bar = u phi, i.e. M1G gains
 *     -S1 A1 d_t(u phi) and the equation gains div(a1 dt d_t(u phi)) (moment and rate variants;
 *     must be 0 for the CDE).
 * Works inside a batch (the batched step follows the variant too).
 * Errors: LBM_ERR_ARG (not an NCDE model, unknown variant, a1 or a cross-diffusion term with the
 *         CDE, non-finite a1). */
lbm_status lbm_model_set_ncde_variant(lbm_model* m, lbm_ncde_variant variant, double a1);

/* The cross-diffusion term of Eq. (GNCDE): A2 = a2 I and D-bar = psi I for a prescribed cell
 * field psi, so that M1G gains -S1 A2 div(D-bar) = -S1 a2 grad psi (Eq. (M-NCDE-6)) and the
 * recovered equation gains div(K2 grad psi) with K2 = dt A2 (the derivation; the printed
 * K2 = dt S1 A2 carries the same slip as the printed K). grad psi is the second-order central
 * difference over the cell spacing c_a dt, read at the 2d neighbours every step; with the rate
 * variant S1 is the per-cell S1(phi). psi[ncells] (grid order, x fastest; host or device per
 * on_device) is copied into the model in the compute dtype and stays until the next call;
 * a2 = 0 removes the term (psi may then be NULL).
 * Errors: LBM_ERR_ARG (not an NCDE model, the CDE variant, non-finite a2, NULL psi with a2 != 0),
 *         LBM_ERR_CUDA. Works inside a batch. */
lbm_status lbm_model_set_ncde_cross_diffusion(lbm_model* m, double a2, const double* psi,
                                              int on_device);

/* The anisotropy term of M2G on the single-speed lattices (Eq. (M2Ga), Sec. 3.4, k = 1): the
 * bracket of M2G gains (delta4 . u) . grad rho, where delta4_aaaa = c_a^2 - 3 c_s^2 (c_s^2 =
 * cs2_eq) and every other component is zero, so the term is (c_a^2 - 3 c_s^2) u_a d_a rho on the
 * normal second moment of axis a. Eq. (M2Ga-1), the default (enable = 0), drops it as O(Ma^3).
 * d_a rho is the second-order central difference, over the cell spacing c_a dt, of the density of
 * the previous step, which the step kernel stores (one field read at the 2d neighbours and one
 * written per cell; FP32 or FP64 as the compute dtype). Enabling takes the density of the current
 * state as the previous one, as init_fields and set_populations do (rho^{-1} = rho^0).
 * Errors: LBM_ERR_ARG (not an NSE model on rD2Q9 / rD3Q27, enable not 0 or 1),
 *         LBM_ERR_CUDA. Works inside a batch (the history then alternates with the batch's steps). */
lbm_status lbm_model_set_m2g_anisotropy(lbm_model* m, int enable);

/* f-bar(t = 0) = f^eq of the given fields (Eq. (feq-1)); for the NCDE phi^{-1} = phi^0.
 * rho_or_phi[ncells], u[d*ncells] (NSE only; ignored and may be NULL for the NCDE). Resets
 * the step counter. Asynchronous when on_device != 0. */
lbm_status lbm_model_init_fields(lbm_model* m, const double* rho_or_phi, const double* u,
                                 int on_device);

/* Set / get the populations f-bar_j(x, t_n) of Eq. (2-3) (pre-collision, after streaming),
 * f[Q*ncells] in FP64. set: for the NCDE phi^{n-1} is set to sum_j f-bar_j. get synchronizes
 * the model's stream when the destination is host memory. */
lbm_status lbm_model_set_populations(lbm_model* m, const double* f, int on_device);
lbm_status lbm_model_get_populations(lbm_model* m, double* f, int on_device);

/* Advance nsteps time steps: per step one fused kernel computes the pull-streaming gather
 * (Eq. (2-2b)), the fields of Eq. (2-4-2) / (2-4-1), the collision of Eq. (2-3) in the Hermite
 * basis with the equilibrium of Eq. (feq-1) and the source moments, and the store.
 * Asynchronous on the model's stream. */
lbm_status lbm_model_step(lbm_model* m, int64_t nsteps);

/* Propagation only (Eq. (2-2b)), no collision: a bit-exact data-movement test mode. */
lbm_status lbm_model_stream_only(lbm_model* m, int64_t nsteps);

/* Macroscopic fields at the current time (Eq. (2-4-2): rho = sum f, u = (sum c f + F/2)/rho;
 * Eq. (2-4-1): phi = sum f) into rho_or_phi[ncells] and u[d*ncells] (u may be NULL; ignored
 * for the NCDE). Synchronizes the stream when the destination is host memory. */
lbm_status lbm_model_read_fields(lbm_model* m, double* rho_or_phi, double* u, int on_device);

/* Global sums over the grid in FP64: out_host[0] = sum_x sum_j f_j,
 * out_host[1 + a] = sum_x sum_j c_ja f_j (a < d). Deterministic (fixed reduction order).
 * Synchronous. Returns LBM_ERR_NONFINITE (with the sums still written) if any is NaN/inf. */
lbm_status lbm_model_conserved_sums(lbm_model* m, double* out_host);

/* The same sums for callers that may not allocate device memory (hosts whose device memory is
 * managed by their own pool allocator or capped by a fixed budget, diagnostics after an
 * out-of-memory error). The paper has no counterpart: this is
 * an interface variant of lbm_model_conserved_sums. Allocates nothing and synchronizes nothing:
 * the reduction scratch is a static device array of 608 x 4 doubles (19,456 bytes) resident on
 * every GPU that loads the library, the result goes to out_dev[4] (device memory, caller-owned,
 * out_dev[0] = mass, out_dev[1 + a] = momentum, unused entries 0), asynchronously on the model's
 * stream. The first call on each device looks up the array's address (and may load device code):
 * make it before any stream capture. All calls share the array and every call rewrites the slots
 * it reads, so no clearing is needed, but calls whose kernels overlap on the GPU race on it.
 * The reduction never needs more than the 608 slots; a build whose reduction grid exceeds the
 * array is rejected with LBM_ERR_ARG, and so is an out_dev that is not device or managed memory
 * of the model's GPU. Non-finite sums are not detected (no host read). The cached address is
 * valid for the device's context: after cudaDeviceReset, reload the library. */
lbm_status lbm_model_conserved_sums_noalloc(lbm_model* m, double* out_dev);

/* Completed time steps since the last init/set; kernels launched by this model so far. */
lbm_status lbm_model_counters(const lbm_model* m, int64_t* steps, int64_t* launches);

/* Wait for the model's stream. */
lbm_status lbm_model_synchronize(lbm_model* m);

lbm_status lbm_model_destroy(lbm_model* m);

/* ------------------------------------------------------------------------------------------
 * Batches: many resident solves advanced together (the paper has no counterpart; this is the
 * execution engine for serving many solves on one GPU)
 * ------------------------------------------------------------------------------------------ */

/* Create an empty batch on the current device. stream: the cudaStream_t every member's kernels
 * run on while it is a member (must be a non-legacy stream so that steps can be captured in a CUDA
 * graph); NULL makes the batch create and own a non-blocking stream. max_solves bounds membership. */
lbm_status lbm_batch_create(void* stream, int max_solves, lbm_batch** out);

/* Add a model (F32, F16_DEV or BF16_DEV storage). The model's stream is synchronized, then the
 * model runs on the batch's stream until it is removed; while a member it is advanced only by
 * lbm_batch_step (lbm_model_step returns LBM_ERR_ARG) but every other model call works (on the
 * batch's stream). Members are grouped by (lattice handle, storage dtype, equation); share one
 * lattice handle between solves of the same lattice setting so that they form one group. Every
 * model setting carries over: the NCDE variants, the cross-diffusion and M2G gradient terms, and
 * distinct rates for the orders >= 4 (such solves form their own groups, with tiles of 128
 * cells, on the CUDA cores). FP64 storage is not batched (LBM_ERR_NOT_IMPLEMENTED). */
lbm_status lbm_batch_add(lbm_batch* b, lbm_model* m);

/* Remove a model. It returns to its own stream, which is made to wait (on the device, through an
 * event) for the batch's steps queued so far: no host synchronization, and any later call on the
 * model sees its state after those steps. The next lbm_batch_step rebuilds the work-lists. */
lbm_status lbm_batch_remove(lbm_batch* b, lbm_model* m);

/* Tile size (cells per thread block) of the batched kernel for one group type: 64, 128 or 256.
 * Default 128. Set by the autotuner (paper_2512_16230_gb300/autotune.py). */
lbm_status lbm_batch_set_tile(lbm_batch* b, lbm_kind kind, lbm_dtype store, lbm_eq eq,
                              int cells_per_tile);

/* Persistent grid of a group's work-list launch: at most `blocks` resident blocks per SM (the
 * grid is that times the SM count, capped by the tile count); 0 (default) takes the occupancy
 * limit of the kernel. A launch-shape knob for autotuning; results do not depend on it.
 * Errors: LBM_ERR_ARG for a negative count. */
lbm_status lbm_batch_set_blocks_per_sm(lbm_batch* b, lbm_kind kind, lbm_dtype store, lbm_eq eq, int blocks);

/* Members of at least `cells` cells (default 2^19) run on the single-solve kernels of
 * lbm_model_step (one launch per step each) instead of the work-list kernel: a grid that large
 * fills the GPU alone, and the single-solve kernels reach a larger share of HBM bandwidth. The
 * results are bitwise the same either way. 0 keeps every member in the work-lists. Errors:
 * LBM_ERR_ARG for a negative threshold. */
lbm_status lbm_batch_set_solo_threshold(lbm_batch* b, int64_t cells);

/* Advance every member by nsteps time steps, asynchronously with respect to the host and in order
 * on the batch's stream. Each step is one persistent launch per group over a tile work-list that
 * covers every cell of every solve of the group (the same per-cell collide-stream arithmetic as
 * lbm_model_step), and one single-solve launch per member above the solo threshold. The work of a
 * call is forked from the batch's stream onto internal streams (one per group, one for the
 * single-solve members), so that groups and large members overlap, and joined back into it before
 * the call returns: anything enqueued on the batch's stream afterwards (an event, a copy, a
 * removal) comes after every member's steps. Chunks of 8 steps are replayed from a captured CUDA
 * graph (one branch per group) once membership has been stable for a whole call. The first call
 * after a membership or parameter change rebuilds the work-lists (a work-list buffer that must grow
 * is reallocated, and cudaFree waits for the device). */
lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* Steps taken, batched launches issued, current number of groups and of tiles. */
lbm_status lbm_batch_counters(const lbm_batch* b, int64_t* steps, int64_t* launches, int* groups,
                              int64_t* tiles);

/* The batch's cudaStream_t (for events and ordering by the caller). */
void* lbm_batch_stream(const lbm_batch* b);

/* Wait for the batch's stream. */
lbm_status lbm_batch_synchronize(lbm_batch* b);

/* Destroy the batch (members are released, not destroyed). */
lbm_status lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_MRT_H */
