// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>

#include "lattices.cuh"
#include "lbm_mrt.h"

// Host-side lattice handle: the FP64 tables built on the GPU by the set-up kernel.
struct lbm_lattice {
  int kind, d, Q, R, rmax;
  int8_t e[lbm::kMaxQ * 3];
  double c[3], cs2[3], free_w[4];
  double w[lbm::kMaxQ];
  double H[lbm::kMaxR * lbm::kMaxQ];
  double N[lbm::kMaxR];
  double T[lbm::kMaxR * lbm::kMaxR];
  // Rows of order >= 4 completing the Q x Q Hermite matrix, W-orthogonal to every row of lower
  // order (graded blocks): even-degree rows first, then odd, each group by order. Values on the
  // lattice, h_order[r] the order and Nh[r] = sum_i w_i Hh_ri^2. high_status: 0 complete,
  // 1 the graded monomials do not reach rank Q, 2 a W-norm vanishes (zero weights).
  int nhigh, high_status;
  int h_order[lbm::kMaxQ];
  double Hh[lbm::kMaxQ * lbm::kMaxQ];
  double Nh[lbm::kMaxQ];
  int device;
};

struct lbm_model {
  const lbm_lattice* lat;
  int eq;
  int64_t n[3];
  int ncells;
  int store, compute;
  cudaStream_t stream;
  void* ws;
  size_t ws_bytes;
  bool owns_ws;
  void* f[2];  // ping-pong population buffers (storage dtype), f[cur] is the current state
  int cur;
  void* phi_prev;   // NCDE: phi at the previous step (compute dtype)
  // single-speed NSE: the density of the previous step for the (delta4 . u) . grad rho term of
  // M2G, Eq. (M2Ga) (two fields in the compute dtype: a step reads rho_hist[hist_cur] at the
  // neighbours and writes rho_hist[hist_cur ^ 1])
  void* rho_hist[2];
  int hist_cur;
  bool m2g_aniso;
  // NCDE: the prescribed field psi of the cross-diffusion term (D-bar = psi I, compute dtype) and
  // its coefficient A2 = a2 I (Eq. (GNCDE)); a2 = 0: no term
  void* psi;
  double a2;
  void* force_tab;  // NSE: F_a as a function of the cell index along axis b (compute dtype)
  double* partials; // reduction scratch of the conservation sums
  double* sums;     // 4 doubles
  double s[lbm::kMaxR];
  double s_high, cs2_eq, rho_ref;
  double s_bulk;  // bulk relaxation rate of Eq. (4-27); <= 0: normal rows relax with their own rates
  double s_order[lbm::kMaxOrder + 1];  // rate of the rows of each order >= 4 (defaults to s_high)
  bool high_explicit;                  // some order >= 4 has a rate other than s_high
  int force_a, force_b, force_k;
  double force_A, force_phase;
  double u_const[3];
  double nonlin;
  int ncde_variant;  // lbm_ncde_variant
  double a1;         // mixed-derivative coefficient A1 = a1 I (Eq. (GNCDE))
  bool tensor_cores; // 16-bit storage: contractions on tcgen05 (k_step_tc)
  bool tc_auto;      // no explicit choice yet: tcgen05 with per-order rates (FP32 or 16-bit storage)
  bool tc_no_issue;  // test hook: k_step_tc issues no matrix product, so its waits run out
  int gather;        // lbm_gather: how the CUDA-core kernel of 16-bit storage gathers (auto, threads, rows)
  bool row_no_copy;  // test hook: the row-staged kernels issue no row copy, so their waits run out
  int* status;       // device status word: non-zero after a device-side wait ran out
  int64_t steps, launches;
  int device;
  lbm_batch* batch;         // batch the model belongs to (its kernels then run on the batch's stream)
  cudaStream_t own_stream;  // the model's stream while it is not in a batch
};

namespace lbm {

// Launch shape of the cell kernels (tuned on GB300; see the kernel notes in mrt_kernels.cuh).
#ifndef LBM_K1_BLOCK
#define LBM_K1_BLOCK 128
#endif
constexpr int kBlock = LBM_K1_BLOCK;  // threads per block of the cell kernels
constexpr int kRedBlocks = 608;      // blocks of the conservation-sum reduction (4 x 152 SMs)
// Largest accepted cell count. Cell indices are 32-bit in the kernels; the margin below 2^31 keeps
// every index a launch or a grid-stride loop can form (cell + one block, cell + the reduction
// grid's stride of kRedBlocks x 256 threads, a tile start + the tile) below 2^31.
constexpr int64_t kMaxCells = (int64_t(1) << 31) - (int64_t(1) << 21);
static_assert(int64_t(kRedBlocks) * 256 < (int64_t(1) << 21), "reduction stride within the index margin");

// Kernel parameters of the time step, passed by value (they live in the constant bank, so
// every table read below is an operand of the arithmetic instruction, not a memory load).
template <class CT>
struct StepParams {
  CT T[kMaxR][kMaxR];  // Hermite rows as monic polynomials of the monomials (physical units)
  CT D[kMaxR];         // monomial scale: mono_k(c_i) = D_k * mono_k(e_i)
  CT invN[kMaxR];      // 1 / N_r
  CT sd[kMaxR];        // s_r - s_high
  CT half[kMaxR];      // 1 - s_r / 2
  CT sdn[3][3];        // normal second-order block: S_n - s_high I (S_n diagonal unless a bulk rate is set)
  CT halfn[3][3];      // I - S_n / 2
  CT w[kMaxQ];
  CT wref[kMaxQ];      // w_i * rho_ref, the offset of deviation storage
  CT wmom_ref[kMaxR];  // rho_ref sum_i w_i mono_k(e_i): moments of the reference state w_i rho_ref
  CT sh_rho_ref;       // s_high * rho_ref
  CT s_high, one_minus_sh, cs2_eq, nonlin_third;
  CT u_const[3];         // NCDE: convection velocity of M1 = u phi (zero for the CDE variant)
  // NCDE variants: per-cell first-order rates (RATE: s_a(phi) = 1 / (kfac_a g(phi) + 1/2),
  // g = 1 + nonlin_rate phi^2) and the CDE source (S_G = sum_a cde_coef_a M1_a, M0G = half0 S_G)
  int ncde_variant;
  CT kfac[3];
  CT nonlin_rate, a1;
  CT cde_coef[3];
  CT half0;
  // A central-difference gradient term (grad_on): gr_a = gscale_a (g(x + e_a) - g(x - e_a)) of the
  // cell field g = grad_in. NSE on rD2Q9 / rD3Q27: g is the previous step's density and
  // gscale_a = (c_a^2 - 3 cs2_eq) / (2 c_a), the delta4 term of M2G (Eq. (M2Ga)); the step writes
  // its own density to rho_out. NCDE: g = psi of the cross diffusion D-bar = psi I and
  // gscale_a = a2 / (2 c_a), the A2 term of M1G (Eq. (M-NCDE-6)).
  int grad_on;
  CT gscale[3];
  const CT* grad_in;
  CT* rho_out;
  int n[3];
  int ncells;
  unsigned div_m[2];     // cell index -> (x, y, z): q = umulhi(v, div_m) >> div_s exactly divides
  int div_s[2];          // by n[0] (slot 0) and n[1] (slot 1) for every v < 2^31
  int force_a, force_b;  // force_b < 0: no body force
  const CT* force_tab;
  static constexpr bool kNcdeVariants = true;
};

// Rows of order >= 4 that relax with their own rates (the full Q x Q collision). The kernel
// adds w_i sum_r h_r(c_i) a_r y_r with y_r = sum_j h_r(c_j) f_j and a_r = -(s_r - s_high) / N_r
// to the reduced-form update; even rows are read at the rest velocity and at the + member of
// each +-e pair, odd rows at the + members (their value at -e is the negative).
template <class CT>
struct HighParams {
  CT he[kMaxHighEven][kMaxPairs + 1];
  CT ho[kMaxHighOdd][kMaxPairs];
  CT ae[kMaxHighEven];
  CT ao[kMaxHighOdd];
};

// Tensor-core kernel parameters: the monomial table mono_k(e_i) (paper's row order) and the
// tile count; status receives 1 if an mbarrier wait ran out.
constexpr int kMaxHigh = kMaxQ - kMaxR;  // rows of order >= 4 (rD3Q53: 33)
struct TcParams {
  int8_t mono[kMaxQ][kMaxR];
  float hrow[kMaxHigh][kMaxQ];  // higher rows on the lattice (one rate per order >= 4)
  float ah[kMaxHigh];           // -(s_r - s_high) / N_r
  int ntiles;
  int* status;
  unsigned wait_limit;  // mbarrier polls before a wait is declared lost
  int no_issue;         // test hook: issue no matrix product (every wait then runs out)
};

// FP32 storage with one rate per order >= 4 on tcgen05 (k_step_tc32_high): the correction of the
// higher rows, w_i sum_r a_r H_r(c_i) sum_j H_r(c_j) f_j, as one dense Q x Q operator applied to
// the pre-collision populations: Delta_i = wg_i sum_j g_ij f_j, with
// g_ij = 2^-k_i sum_r a_r H_r(c_i) H_r(c_j) (k_i brings the row's max |g_ij| into [1, 2)) and
// wg_i = 2^k_i w_i.
struct Tc32Params {
  float g[kMaxQ][kMaxQ];
  float wg[kMaxQ];
  int ntiles;
  int* status;
  unsigned wait_limit;  // mbarrier polls before a wait is declared lost
  int no_issue;         // test hook: issue no matrix product (every wait then runs out)
};

// Row-staged collide-stream kernel (16-bit storage, row_kernels.cuh): row buffers of kRowPitch
// cells per population (the largest n_x; one cell per thread of a kRowThreads CTA), up to
// kRowMaxStages buffers behind kRowBarBytes of mbarriers and counters.
constexpr int kRowPitch = 256;
constexpr int kRowThreads = kRowPitch;
constexpr int kRowMaxStages = 8;
constexpr int kRowBarBytes = 256;
struct RowParams {
  // byte offset from the start of row r of the population arrays to the pull-source row of
  // population i, 2 (i N - (e_iy + e_iz n_y) n_x), valid for rows away from the y and z faces
  int64_t src_off[kMaxQ];
  int8_t ey[kMaxQ], ez[kMaxQ];  // y and z velocity components (source rows next to a face)
  int nrows;                    // n_y n_z
  int stages;                   // row buffers per CTA
  uint32_t stage_bytes;         // Q * pitch * 2
  int* status;
  unsigned wait_limit;          // mbarrier polls before a wait is declared lost
  int no_copy;                  // test hook: issue no row copy (every wait then runs out)
};
struct RowPlan {
  int grid;
  size_t smem;
  RowParams rp;
  bool tensor;  // the tensor-core kernel (k_step_rows_tc) for the collide steps
  bool high;    // with the rows of order >= 4 at their own rates (tensor-core kernel only)
  TcParams tp;
};
template <int KIND>
struct RowLaunch {
  // false when the kernel does not apply (storage not 16-bit, n_x not a multiple of 8 or above the
  // pitch, or the shared memory cannot hold three row buffers); `tensor`: the tensor-core kernel,
  // `high`: with one rate per order >= 4 (needs `tensor`)
  static bool plan(const lbm_model* m, RowPlan* out, bool tensor = false, bool high = false);
  static lbm_status configure(const lbm_model* m, const RowPlan& plan, bool collide);
  static lbm_status launch(const lbm_model* m, const RowPlan& plan, const StepParams<float>& p, const void* fin,
                           void* fout, float* phi, bool collide);
};

// Multiply-high division by a runtime divisor 2 <= d < 2^31, exact for numerators below 2^31:
// with s = ceil(log2 d) and m = ceil(2^(31+s) / d) < 2^32, floor(v / d) = (v m / 2^32) >> (s-1).
inline void division_magic(unsigned d, unsigned* m, int* shift) {
  int s = 0;
  while ((1ull << s) < d) ++s;
  *m = unsigned(((1ull << (31 + s)) + d - 1) / d);
  *shift = s - 1;
}

// Parameters of the generic (lattice-agnostic, non-hot) kernels.
struct GenParams {
  int Q, d, n[3], ncells;
  int8_t e[kMaxQ][3];
  double c[3];
  double wref[kMaxQ];
  double cde_half[3];  // NCDE CDE variant: phi = sum f + sum_a cde_half_a sum_i c_ia f_i
  int force_a, force_b;
  const void* force_tab;
};

// Per-velocity tables of the generic kernels in their compute dtype (c_ia and w_i rho_ref), so
// that no FP64 arithmetic runs per population when the model computes in FP32.
template <class CT>
struct GenTables {
  CT ce[kMaxQ][3];
  CT wref[kMaxQ];
};

// Storage codecs: FP64/FP32 store f itself; BF16/FP16 store the deviation f - w_i rho_ref.
template <class ST>
struct Codec;
template <>
struct Codec<double> {
  template <class CT> __device__ __forceinline__ static CT dec(double v, CT) { return CT(v); }
  template <class CT> __device__ __forceinline__ static double enc(CT v, CT) { return double(v); }
};
template <>
struct Codec<float> {
  template <class CT> __device__ __forceinline__ static CT dec(float v, CT) { return CT(v); }
  template <class CT> __device__ __forceinline__ static float enc(CT v, CT) { return float(v); }
};
template <>
struct Codec<__nv_bfloat16> {
  template <class CT> __device__ __forceinline__ static CT dec(__nv_bfloat16 v, CT base) {
    return CT(__bfloat162float(v)) + base;
  }
  template <class CT> __device__ __forceinline__ static __nv_bfloat16 enc(CT v, CT base) {
    return __float2bfloat16_rn(float(v - base));
  }
};
template <>
struct Codec<__half> {
  template <class CT> __device__ __forceinline__ static CT dec(__half v, CT base) {
    return CT(__half2float(v)) + base;
  }
  template <class CT> __device__ __forceinline__ static __half enc(CT v, CT base) {
    return __float2half_rn(float(v - base));
  }
};

// Deviation storage read and written as deviations (no reference offset).
template <class ST>
struct RawCodec;
template <>
struct RawCodec<__nv_bfloat16> {
  __device__ __forceinline__ static float dec(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 enc(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct RawCodec<__half> {
  __device__ __forceinline__ static float dec(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half enc(float v) { return __float2half_rn(v); }
};
template <class ST>
constexpr bool is_deviation_storage() {
  return std::is_same<ST, __nv_bfloat16>::value || std::is_same<ST, __half>::value;
}

inline size_t dtype_bytes(int dt) { return dt == LBM_F64 ? 8 : dt == LBM_F32 ? 4 : 2; }

// Error reporting (thread-local message behind lbm_last_error).
lbm_status set_error(lbm_status st, const std::string& msg);
lbm_status cuda_error(cudaError_t err, const char* what);

// ---- Batched execution (one launch advances every solve of a group by one step) ----

// Lattice tables shared by every solve of a group (kernel parameter: constant bank).
template <class CT>
struct BatchTables {
  CT T[kMaxR][kMaxR];
  CT D[kMaxR];
  CT invN[kMaxR];
  CT w[kMaxQ];
  CT wref[kMaxQ];
  CT wmom_ref[kMaxR];
};

// Per-solve data of a batched step (device array; each block stages its solve's entry in shared
// memory). f[k] is the input of a step launched with parity k and f[k ^ 1] its output.
template <class CT>
struct __align__(16) SolveDesc {
  CT sd[kMaxR];
  CT half[kMaxR];
  CT sdn[3][3];
  CT halfn[3][3];
  CT s_high, one_minus_sh, sh_rho_ref, cs2_eq, nonlin_third;
  CT u_const[3];
  int n[3];
  int ncells;
  unsigned div_m[2];
  int div_s[2];
  int force_a, force_b;
  const CT* force_tab;
  void* f[2];
  CT* phi;
  // NCDE variants (as in StepParams)
  int ncde_variant;
  CT kfac[3];
  CT nonlin_rate, a1;
  CT cde_coef[3];
  CT half0;
  // gradient terms (as in StepParams): a step launched with parity k reads grad_in[k] and, for the
  // delta4 term of M2G, writes its density to rho_out[k]
  int grad_on;
  CT gscale[3];
  const CT* grad_in[2];
  CT* rho_out[2];
};

struct Tile {
  int solve;  // index into the group's descriptor array
  int cell0;  // first cell of the tile (tiles are blockDim cells long, the last one ragged)
};

// A group of solves advanced by one batched launch per step.
struct BatchGroup {
  int kind, store, eq, block;
  int high;         // the solves have one rate per order >= 4 (k_step_batch_high, tiles of kBlock cells)
  const lbm_lattice* lat;
  void* tables;     // host copy of BatchTables<CT>
  void* d_desc;     // device SolveDesc<CT>[nsolves]
  void* d_high;     // device HighParams<CT>[nsolves] (high groups)
  Tile* d_tiles;    // device work-list
  int nsolves, ntiles, grid;
};

template <int KIND>
struct BatchLaunch {
  static lbm_status launch(const BatchGroup& g, int parity, cudaStream_t stream);
  static lbm_status occupancy(int store, int eq, int block, int high, int* blocks_per_sm);
};

// Per-lattice launchers, defined in the k_<lattice>.cu translation units.
template <int KIND>
struct Launch {
  static lbm_status step(lbm_model* m, int64_t nsteps, bool collide);
  static lbm_status init(lbm_model* m, const double* rho_or_phi, const double* u);
};

// Generic kernels (aux_kernels.cu).
lbm_status gen_params(const lbm_model* m, GenParams* gp);
lbm_status launch_gather(lbm_model* m, double* out);          // f-bar(x) from the stored array
lbm_status launch_scatter(lbm_model* m, const double* in);    // stored array from f-bar(x)
lbm_status launch_fields(lbm_model* m, double* rho, double* u);
lbm_status launch_sums(lbm_model* m);                          // into m->sums (device)
lbm_status launch_phi_from_populations(lbm_model* m);          // NCDE: phi_prev = sum f-bar
lbm_status launch_density_history(lbm_model* m);               // single-speed NSE: rho_hist[hist_cur] = sum f-bar
lbm_status launch_to_compute(lbm_model* m, const double* src, void* dst);  // a cell field in the compute dtype
// The conservation-sum kernels with caller-provided reduction scratch (partial_slots x 4
// doubles, at least kRedBlocks slots) and result (4 doubles, device memory).
lbm_status launch_sums_into(lbm_model* m, double* partials, int partial_slots, double* out);

// Batches (batch.cu): a parameter change of a member invalidates the batch's captured work.
void batch_mark_dirty(lbm_batch* b);

// FP64 lattice set-up on the GPU (setup_fp64.cu).
lbm_status setup_lattice_fp64(lbm_lattice* lat);

// Host-side construction of the step parameters from a model.
template <class CT>
void make_step_params(const lbm_model* m, StepParams<CT>* p);
template <class CT>
void make_high_params(const lbm_model* m, HighParams<CT>* hp);
// true when some row of order >= 4 relaxes with a rate other than s_high
bool has_high_rates(const lbm_model* m);
void make_tc_params(const lbm_model* m, TcParams* tp);
void make_tc32_params(const lbm_model* m, Tc32Params* tp);
int tc_grid(const lbm_model* m, int ntiles, const void* kernel, int ctas_per_sm, size_t smem_bytes);

}  // namespace lbm
