// Internal declarations of the GB300 w-stacking w-projection library.
//
// Layout in HBM (one plan):
//   VisRec<T>[n_kept]   visibility records sorted by (stack, uv tile), one
//                       32 B (FP32) or 48 B (FP64) record per visibility:
//                       fractional grid position, integer base, w offset,
//                       weight and support;
//   perm[n_kept]        caller index of each sorted record, bit 31 = folded;
//   omn_pix[N*N]        1 - n(l, m) per pixel (FP64, for the chirp phase);
//   corr_pix[N*N]       1 / (g(du |l|) n(l, m)) per pixel (precision T);
//   node tables         per panel count P = 1..128: 1 - n(r_j) (FP64) and
//                       w 2 pi h g(r_j) r_j (T: the Kronrod weight, and the
//                       Gauss weight in FP32 or the Kronrod-minus-Gauss
//                       weight in FP64) at the 31 P Gauss-Kronrod nodes;
//   tap order           per even support J_w, its J_w^2 taps sorted by
//                       distance from the box centre (uint16 a | b << 8);
//   grids               padded complex grids of one group of stacks at a
//                       time (as many as fit max_grid_mib), reused by every
//                       group;
//   counters            work-queue heads and quadrature statistics;
//   fixed-point grids   grid_deterministic = 1 only: two int64 per cell of
//                       the group's grids, the gridding sums before they
//                       are rounded into the complex grids.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/phi.h"

namespace phi {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr float kPiF = 3.14159265358979323846f;

// Gauss-Kronrod 15/31 nodes per panel; panel counts 1..kMaxPanels, the node
// tables holding every partition (panel count P at offset 31 P (P - 1) / 2).
constexpr int kNodesPerPanel = 31;
constexpr int kMaxPanels = 128;
__host__ __device__ inline int64_t panel_table_offset(int npan) {
  return kNodesPerPanel * static_cast<int64_t>(npan) * (npan - 1) / 2;
}
__host__ __device__ inline int panel_count_for(float want) {
  // want may be NaN or huge: clamp without relying on the conversion
  if (!(want > 1.0f)) return 1;
  if (want >= static_cast<float>(kMaxPanels)) return kMaxPanels;
  return static_cast<int>(ceilf(want));
}

// Largest number of visibility records in one uv-tile work item, and in one
// w-row work item of the table path's row staging.
constexpr int kItemRecords = 128;
constexpr int kRowItemRecords = 1024;

// Panels evaluated per batch out of the per-warp shared node buffer.
constexpr int kPanelBatch = 8;
constexpr int kNodeBatch = kNodesPerPanel * kPanelBatch;

template <typename T> struct Cplx;
template <> struct Cplx<float> { typedef float2 type; };
template <> struct Cplx<double> { typedef double2 type; };

template <typename T>
struct __align__(16) VisRec;

template <>
struct __align__(16) VisRec<float> {
  float fu, fv;      // u/du - bu, v/du - bv, in [0, 1)
  int32_t bu, bv;    // floor(u/du), floor(v/du)
  double dw;         // w - wbar_k (FP64: it multiplies the chirp phase)
  float weight;      // W_i
  uint16_t jw;       // support J_w (even, <= 256)
  uint16_t stack;    // w-stack k
};

template <>
struct __align__(16) VisRec<double> {
  double fu, fv;
  double dw;
  double weight;
  int32_t bu, bv;
  int32_t jw;
  int32_t stack;
};

// Shared per-node integrand values of one visibility, with the Kronrod
// weight (k) and the Kronrod-minus-Gauss weight (d) folded in.
template <typename T> struct NodeVal;
template <> struct __align__(16) NodeVal<float> { float kr, ki, dr, di; };
template <> struct __align__(16) NodeVal<double> { double kr, ki, dr, di; };

// Radial interpolation mode (PHI_KERNEL_RADIAL): Chebyshev points per piece
// of [0, rho_max], by precision (interpolation error ~1e-7 and ~4e-14 of
// K(0) at pieces of 2 / R pixels).
template <typename T> struct RadialN;
template <> struct RadialN<float> { static constexpr int n = 16; };
template <> struct RadialN<double> { static constexpr int n = 24; };

// Kernel-side view of the radial mode's tables: piece width L (grid pixels)
// and 1 / L; x1[j] = (1 + cos(pi (j + 1/2) / n)) / 2, the Chebyshev points
// mapped to [0, 1]; dct[j n + m] = cos(pi m (j + 1/2) / n); buf = complex
// values of series storage per warp (pieces x (n + 1)).
template <typename T>
struct RadialView {
  T L, inv_L;
  const T* x1;
  const T* dct;
  int buf;
};

// Deterministic gridding target (grid_deterministic = 1): per grid cell two
// int64 (re, im) holding the cell's sum in units of 2^-exp[0], so that the
// sum does not depend on the order of its additions; exp[1] != 0 marks a
// non-finite visibility.  cells == nullptr: gridding adds its values to the
// complex grid with FP atomics instead.
struct FixedGrid {
  unsigned long long* cells;
  const int* exp;
};

// Kernel-side constants of one plan.
struct QuadParams {
  double R;               // window radius (r units)
  float Rf;               // the same, for the panel-count estimate
  float chirp_coeff;      // local chirp frequency at r = R per unit |dw|
  float inv_cycles;       // 1 / (integrand cycles per panel)
  float tol_rel, tol_abs;
  int max_refine;         // panel-count doublings allowed
  int npad;
  const double* node_omn;  // 1 - n(r_j) per node, all panel counts
  const void* node_hk;     // w_K(j) 2 pi h g(r_j) r_j per node (T)
  const void* node_hd;     // w_G(j) (FP32) or w_K(j) - w_G(j) (FP64), times 2 pi h g(r_j) r_j
  const uint16_t* tap_order;  // per even J_w: taps (a | b << 8) by distance from the box centre
  const int32_t* tap_off;     // offset of the list for J_w = 2 i + 2 at index i
  FixedGrid fx;               // gridding target of deterministic plans
};

struct Plan {
  phi_plan_desc d;
  int N = 0, npad = 0, K = 0;
  double dl = 0, du = 0, R = 0, beta = 0, i0beta = 0, l_win = 0, n_win = 0, c_support = 0;
  double cycles_per_panel = 0;
  int64_t M = 0, n_kept = 0, n_dropped = 0;
  int kmeans_sweeps = 0;
  int max_jw = 0;
  std::vector<double> wbar;
  std::vector<int64_t> stack_off;   // K + 1 offsets into the sorted records
  std::vector<int32_t> stack_jw;    // per-stack support (max under the per-vis rule)
  // device memory
  void* recs = nullptr;
  uint32_t* perm = nullptr;
  double* omn_pix = nullptr;
  void* corr_pix = nullptr;
  double* node_omn = nullptr;
  void* node_hk = nullptr;
  void* node_hd = nullptr;
  uint16_t* tap_order = nullptr;
  int32_t* tap_off = nullptr;
  void* grid = nullptr;                // group * Npad^2 complex: grids of one stack group
  int group = 1;                        // stacks whose grids are resident together
  std::vector<int64_t> group_off;       // groups: stacks group_stacks[group_off[g] .. group_off[g+1])
  std::vector<int32_t> group_stacks;    // the stacks with visibilities, in order
  int32_t* group_stacks_dev = nullptr;
  int32_t* stack_slot_dev = nullptr;    // slot of each stack within its group
  double* wbar_dev = nullptr;
  cufftHandle fft_batch = 0;            // `group` transforms in one call
  bool fft_batch_ok = false;
  // [0..K) work heads, [K] unconverged taps, [K+1] taps, [K+2] wkernel misses,
  // [K+3] tap-node evaluations
  unsigned long long* counters = nullptr;
  // per-stage timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, size_t>> ev_pending;  // (stage, index of start event)
  double stage_ms[PHI_NUM_STAGES] = {0};
  int64_t stage_launches[PHI_NUM_STAGES] = {0};
  cufftHandle fft = 0;
  bool fft_ok = false;
  int64_t device_bytes = 0;
  int num_sms = 0;
  // pre-sampled w-planes (PHI_KERNEL_TABLE): (nw - 1) x nr pairs
  // {K(j h_w, i h_rho), K((j + 1) h_w, i h_rho)} of precision T
  void* table = nullptr;
  int64_t table_nr = 0, table_nw = 0;
  double table_hr = 0, table_hw = 0;
  std::vector<double> stack_maxabs;   // largest |w - wbar_k| of each stack's kept visibilities
  // work items of the table path's staged kernels.  grid_staging 1: item i
  // covers sorted records [item_start[2 i], item_start[2 i + 1]), all in the
  // uv tile item_key[i] (low 24 bits: tile_v * tiles_per_row + tile_u), at
  // most kItemRecords; grid_staging 2: the records row_idx[item_start[2 i]
  // .. item_start[2 i + 1]), all on w-row item_key[i] (low 24 bits), at most
  // kRowItemRecords; the top 8 bits of a key hold the stack
  int32_t* item_start = nullptr;
  uint32_t* item_key = nullptr;
  uint32_t* row_idx = nullptr;          // kept records sorted by (stack, w-row)
  std::vector<int64_t> stack_item_off;  // K + 1 offsets into the items
  std::vector<uint8_t> stack_staged;    // table path: stage this stack's grid tiles
  int tile = 32;
  int tiles_per_row = 0;
  // radial interpolation mode (PHI_KERNEL_RADIAL): tables of precision T
  // (x1[n] then dct[n * n]), piece width, series storage per warp
  void* radial_tab = nullptr;
  double radial_L = 0;
  int radial_buf = 0;
  // deterministic gridding (grid_deterministic = 1): fixed-point sums of the
  // group's grids (group * Npad^2 * 2 int64), the largest |W_i y_i| term
  // factor of a call (double bits), the exponent and non-finite flag, and
  // max over panel counts of sum_j |w_K(j) 2 pi h g(r_j) r_j|, which bounds
  // every tap |[GC]| the quadrature can return
  unsigned long long* fx_cells = nullptr;
  unsigned long long* fx_max = nullptr;
  int* fx_exp = nullptr;
  double kernel_bound = 0;

  QuadParams quad() const {
    QuadParams q;
    q.R = R;
    q.Rf = static_cast<float>(R);
    q.chirp_coeff = static_cast<float>(c_support);
    q.inv_cycles = static_cast<float>(1.0 / cycles_per_panel);
    q.tol_rel = d.quad_rel_tol;
    q.tol_abs = d.quad_abs_tol;
    q.max_refine = d.max_refine;
    q.npad = npad;
    q.node_omn = node_omn;
    q.node_hk = node_hk;
    q.node_hd = node_hd;
    q.tap_order = tap_order;
    q.tap_off = tap_off;
    q.fx.cells = fx_cells;
    q.fx.exp = fx_exp;
    return q;
  }
};

#define PHI_CUDA_TRY(expr)                       \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) {                     \
      (void)cudaGetLastError();                  \
      return e_ == cudaErrorMemoryAllocation ? PHI_ERR_OOM : PHI_ERR_CUDA; \
    }                                            \
  } while (0)

// Calls that read a result back synchronise their stream, which is not
// allowed while the stream is being captured into a graph: refuse them.
#define PHI_TRY_NOT_CAPTURING(stream)                                   \
  do {                                                                  \
    cudaStreamCaptureStatus cs_ = cudaStreamCaptureStatusNone;          \
    PHI_CUDA_TRY(cudaStreamIsCapturing((stream), &cs_));                \
    if (cs_ != cudaStreamCaptureStatusNone) return PHI_ERR_ARG;         \
  } while (0)

// Kernel-side view of the pre-sampled w-planes.
template <typename T>
struct TableView {
  const void* pairs;   // C2<T> [(nw - 1) * nr]
  int64_t nr, nw;
  T inv_hr, inv_hw;
  FixedGrid fx;        // gridding target of deterministic plans
};

// Stage timing (no-ops unless enabled): returns the start-event index or -1.
long timer_begin(Plan& p, cudaStream_t s);
void timer_end(Plan& p, long idx, int stage, cudaStream_t s);

// Launchers implemented in phi_ops.cu.
int launch_node_tables(Plan& p, cudaStream_t s);
int launch_pixel_tables(Plan& p, cudaStream_t s);
int build_kernel_table(Plan& p, cudaStream_t s);
int build_radial_tables(Plan& p, cudaStream_t s);
int compute_kernel_bound(Plan& p, double* scratch, cudaStream_t s);  // scratch: kMaxPanels doubles

}  // namespace phi

// The opaque handle of the C ABI is the plan itself.
struct phi_plan : public phi::Plan {};
