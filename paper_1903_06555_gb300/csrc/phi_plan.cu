// Plan construction for the GB300 w-stacking w-projection operator:
// conjugate fold (Sec. 3.3), k-means w-stacking (Algorithm 1), per-stack
// centres, drop test, support J_w, split of u/du into an integer base and a
// fraction, sort by (stack, uv tile), per-pixel and per-node tables, cuFFT.
//
// All per-visibility work runs on the device.  The k-means sums are exact
// integer sums of a fixed-point image of w, independent of their order, so a
// plan is bit-reproducible run to run.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "phi_internal.cuh"
#include "kmeans_assign.cuh"
#include "table_index.cuh"

namespace phi {

int set_kernel_smem_limits();

namespace {

constexpr int kPlanThreads = 256;
constexpr int kSweepBatch = 8;   // k-means sweeps launched per host round trip

// Fold and extract w.  flag = 1 when the visibility was reflected.
// Non-finite baselines are counted (the plan then refuses them).
__global__ void fold_kernel(const double* __restrict__ uvw, int64_t M, int fold,
                            double* __restrict__ w_out, uint8_t* __restrict__ flag,
                            double* __restrict__ part_min, double* __restrict__ part_max,
                            unsigned long long* __restrict__ n_bad) {
  __shared__ double smin[kPlanThreads], smax[kPlanThreads];
  double lo = INFINITY, hi = -INFINITY;
  unsigned long long bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    double w = uvw[3 * i + 2];
    if (!isfinite(uvw[3 * i]) || !isfinite(uvw[3 * i + 1]) || !isfinite(w)) {
      ++bad;
      w = 0.0;
    }
    uint8_t f = (fold && w < 0.0) ? 1 : 0;
    if (f) w = -w;
    w_out[i] = w;
    flag[i] = f;
    lo = fmin(lo, w);
    hi = fmax(hi, w);
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part_min[blockIdx.x] = smin[0];
    part_max[blockIdx.x] = smax[0];
  }
  if (bad) atomicAdd(n_bad, bad);
}

// One sweep of Algorithm 1: every visibility's nearest centre, and per block
// the fixed-point limb sums and member counts of each stack.  Block b owns
// the contiguous range [b*chunk, (b+1)*chunk); each warp takes 32 consecutive
// visibilities at a time (the next group's w loaded ahead), sums the limbs of
// every stack present among them with warp reductions and adds them to its
// own accumulators in shared memory (lane l holds limb l); the block adds
// its warps' accumulators at the end.  Integer sums: exact and
// order-independent.  `part` = 0 skips the sums; a set `*done` (the
// iteration has converged) makes the launch a no-op.
__global__ void kmeans_sweep_kernel(const double* __restrict__ w, int64_t M, int64_t chunk,
                                    const double* __restrict__ centres, int K, int S,
                                    int32_t* __restrict__ stack,
                                    unsigned long long* __restrict__ part,
                                    const int* __restrict__ done) {
  if (done && *done) return;
  extern __shared__ unsigned long long sm_u64[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  unsigned long long* wacc = sm_u64;                                 // [nwarps][K][kAcc]
  double* c = reinterpret_cast<double*>(wacc + static_cast<size_t>(nwarps) * K * kAcc);
  float* cf = reinterpret_cast<float*>(c + K);
  float* ce = cf + K;
  for (int q = threadIdx.x; q < K; q += blockDim.x) {
    const double cq = centres[q];
    c[q] = cq;
    cf[q] = static_cast<float>(cq);
    ce[q] = km_centre_err(cf[q]);
  }
  for (int q = threadIdx.x; q < nwarps * K * kAcc; q += blockDim.x) wacc[q] = 0ULL;
  __syncthreads();
  unsigned long long* my = wacc + static_cast<size_t>(warp) * K * kAcc;
  const int64_t b0 = blockIdx.x * chunk;
  const int64_t b1 = min(M, b0 + chunk);
  const int64_t step = 32 * (int64_t)nwarps;
  int64_t base = b0 + 32 * (int64_t)warp;
  double wn = (base + lane < b1) ? w[base + lane] : 0.0;
  for (; base < b1; base += step) {
    const int64_t i = base + lane;
    const bool valid = i < b1;
    const double wi = wn;
    if (base + step + lane < b1) wn = w[base + step + lane];
    int s = -1;
    long long v = 0;
    if (valid) {
      s = nearest_centre(wi, c, cf, ce, K);
      stack[i] = s;
      v = w_fixed(wi, S);
    }
    if (!part) continue;
    unsigned limb[kLimbs];
#pragma unroll
    for (int l = 0; l < kLimbs; ++l) limb[l] = w_limb(v, l);
    unsigned rem = __ballot_sync(0xffffffffu, valid);
    while (rem) {
      const int sq = __shfl_sync(0xffffffffu, s, __ffs(rem) - 1);
      const bool in = s == sq;
      const unsigned mem = __ballot_sync(0xffffffffu, in);
      unsigned mine = static_cast<unsigned>(__popc(mem));   // lane kLimbs: the count
#pragma unroll
      for (int l = 0; l < kLimbs; ++l) {
        const unsigned t = __reduce_add_sync(0xffffffffu, in ? limb[l] : 0u);
        if (lane == l) mine = t;
      }
      if (lane < kAcc) my[sq * kAcc + lane] += mine;
      rem &= ~mem;
    }
  }
  if (!part) return;
  __syncthreads();
  for (int q = threadIdx.x; q < K * kAcc; q += blockDim.x) {
    unsigned long long t = 0;
    for (int wp = 0; wp < nwarps; ++wp) t += wacc[static_cast<size_t>(wp) * K * kAcc + q];
    part[static_cast<int64_t>(blockIdx.x) * K * kAcc + q] = t;
  }
}

// Centre update: one warp per stack sums the blocks' limb sums and counts
// (exact integer sums), rebuilds the 96-bit fixed-point total, and sets
// wbar_q = total 2^-S / count, or 0 for an empty stack (Algorithm 1); then
// the convergence measure mean_q |new - old| / max(|old|, eps).
// out[0..K) new centres, out[K..2K) counts, out[2K] measure.  state[0]
// (done) is set once the measure falls below tol or state[1] (sweeps, counted
// here) reaches max_iter; a launch after that is a no-op.
__global__ void kmeans_update_kernel(const unsigned long long* __restrict__ part, int nblocks,
                                     int K, int S, double eps, double tol, int max_iter,
                                     double* __restrict__ centres, double* __restrict__ out,
                                     int* __restrict__ state) {
  if (state[0]) return;
  extern __shared__ double rel[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int q = warp; q < K; q += nwarps) {
    unsigned long long sum[kAcc];
#pragma unroll
    for (int l = 0; l < kAcc; ++l) sum[l] = 0ULL;
    for (int b = lane; b < nblocks; b += 32) {
      const unsigned long long* pb = part + (static_cast<int64_t>(b) * K + q) * kAcc;
#pragma unroll
      for (int l = 0; l < kAcc; ++l) sum[l] += pb[l];
    }
#pragma unroll
    for (int l = 0; l < kAcc; ++l)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum[l] += __shfl_xor_sync(0xffffffffu, sum[l], o);
    if (lane == 0) {
      const double total = fixed_total(sum, S);
      const double n = static_cast<double>(sum[kLimbs]);
      const double old = centres[q];
      const double nc = sum[kLimbs] > 0 ? total / n : 0.0;
      rel[q] = fabs(nc - old) / fmax(fabs(old), eps);
      centres[q] = nc;
      out[q] = nc;
      out[K + q] = n;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int k = 0; k < K; ++k) d += rel[k];
    d /= K;
    out[2 * K] = d;
    const int sweeps = state[1] + 1;
    state[1] = sweeps;
    if (d < tol || sweeps >= max_iter) state[0] = 1;
  }
}

// Per visibility after clustering: w offset, drop test, sort key, and the
// per-stack largest |dw| and kept count (order-independent atomics: integer
// adds and max on the bit pattern of non-negative doubles).
__global__ void classify_kernel(const double* __restrict__ uvw, const uint8_t* __restrict__ flag,
                                const double* __restrict__ w_fold,
                                const int32_t* __restrict__ stack,
                                const double* __restrict__ centres, int64_t M, int K, double du,
                                int npad, int tile, int tiles_per_row,
                                uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                unsigned long long* __restrict__ maxabs_bits,
                                unsigned long long* __restrict__ kept) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double sgn = flag[i] ? -1.0 : 1.0;
    const double up = sgn * uvw[3 * i] / du;
    const double vp = sgn * uvw[3 * i + 1] / du;
    const int s = stack[i];
    const double h = 0.5 * npad;
    const bool drop = !(up >= -h && up < h && vp >= -h && vp < h);
    uint32_t key;
    if (drop) {
      key = static_cast<uint32_t>(K) << 24;
    } else {
      const int64_t bu = static_cast<int64_t>(floor(up)) + npad / 2;
      const int64_t bv = static_cast<int64_t>(floor(vp)) + npad / 2;
      const uint32_t tu = static_cast<uint32_t>(bu / tile), tv = static_cast<uint32_t>(bv / tile);
      key = (static_cast<uint32_t>(s) << 24) | (tv * tiles_per_row + tu);
      const double a = fabs(w_fold[i] - centres[s]);
      atomicMax(maxabs_bits + s, static_cast<unsigned long long>(__double_as_longlong(a)));
      atomicAdd(kept + s, 1ULL);
    }
    keys[i] = key;
    vals[i] = static_cast<uint32_t>(i);
  }
}

template <typename T>
__global__ void records_kernel(const double* __restrict__ uvw, const uint8_t* __restrict__ flag,
                               const double* __restrict__ w_fold,
                               const int32_t* __restrict__ stack,
                               const double* __restrict__ centres,
                               const double* __restrict__ weights,
                               const uint32_t* __restrict__ sorted_vals, int64_t n_kept,
                               double du, int J, double c_support, int per_vis,
                               const int32_t* __restrict__ stack_jw, VisRec<T>* __restrict__ recs,
                               uint32_t* __restrict__ perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_kept;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t o = sorted_vals[i];
    const double sgn = flag[o] ? -1.0 : 1.0;
    const double up = sgn * uvw[3 * (int64_t)o] / du;
    const double vp = sgn * uvw[3 * (int64_t)o + 1] / du;
    const int s = stack[o];
    const double dw = w_fold[o] - centres[s];
    const double bu = floor(up), bv = floor(vp);
    VisRec<T> r;
    r.fu = static_cast<T>(up - bu);
    r.fv = static_cast<T>(vp - bv);
    r.bu = static_cast<int32_t>(bu);
    r.bv = static_cast<int32_t>(bv);
    r.dw = dw;
    r.weight = static_cast<T>(weights ? weights[o] : 1.0);
    r.jw = static_cast<decltype(r.jw)>(per_vis ? J + 2 * static_cast<int32_t>(ceil(fabs(dw) * c_support))
                                               : stack_jw[s]);
    r.stack = static_cast<decltype(r.stack)>(s);
    recs[i] = r;
    perm[i] = o | (flag[o] ? 0x80000000u : 0u);
  }
}

// Tile segmentation of the sorted records: flag the first record of each
// (stack, tile) key, then scatter the starts and keys of the tiles.
__global__ void tile_flag_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                 uint32_t* __restrict__ flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void tile_scatter_kernel(const uint32_t* __restrict__ keys,
                                    const uint32_t* __restrict__ flag,
                                    const uint32_t* __restrict__ pos, int64_t n,
                                    int32_t* __restrict__ start, uint32_t* __restrict__ key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) {
      start[pos[i]] = static_cast<int32_t>(i);
      key[pos[i]] = keys[i];
    }
}

// Table path, w-row staging: per kept record (sorted order) the key
// (stack, w-row of its |dw|), the row computed in precision T exactly as the
// table kernels compute it, and the record's index.
template <typename T>
__global__ void row_key_kernel(const VisRec<T>* __restrict__ recs, int64_t n, T inv_hw,
                               int last_row, uint32_t* __restrict__ keys,
                               uint32_t* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int row = table_w_row(table_w_scaled(static_cast<T>(fabs(recs[i].dw)), inv_hw), last_row);
    keys[i] = (static_cast<uint32_t>(recs[i].stack) << 24) | static_cast<uint32_t>(row);
    vals[i] = static_cast<uint32_t>(i);
  }
}

struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename X>
  cudaError_t alloc(X** p, size_t count) {
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, std::max<size_t>(count, 1) * sizeof(X));
    if (e == cudaSuccess) {
      ptrs.push_back(raw);
      *p = static_cast<X*>(raw);
    }
    return e;
  }
};

void free_plan(Plan* p) {
  if (!p) return;
  if (p->fft_ok) cufftDestroy(p->fft);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  cudaFree(p->recs);
  cudaFree(p->perm);
  cudaFree(p->omn_pix);
  cudaFree(p->corr_pix);
  cudaFree(p->node_omn);
  cudaFree(p->node_hk);
  cudaFree(p->node_hd);
  cudaFree(p->tap_order);
  cudaFree(p->tap_off);
  cudaFree(p->radial_tab);
  cudaFree(p->grid);
  cudaFree(p->counters);
  cudaFree(p->table);
  cudaFree(p->item_start);
  cudaFree(p->item_key);
  cudaFree(p->row_idx);
  cudaFree(p->group_stacks_dev);
  cudaFree(p->stack_slot_dev);
  cudaFree(p->wbar_dev);
  cudaFree(p->fx_cells);
  cudaFree(p->fx_max);
  cudaFree(p->fx_exp);
  if (p->fft_batch_ok) cufftDestroy(p->fft_batch);
}

template <typename X>
cudaError_t owned_alloc(Plan& p, X** ptr, size_t count) {
  void* raw = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(X);
  cudaError_t e = cudaMalloc(&raw, bytes);
  if (e == cudaSuccess) {
    *ptr = static_cast<X*>(raw);
    p.device_bytes += static_cast<int64_t>(bytes);
  }
  return e;
}

#define PHI_TRY(expr)             \
  do {                            \
    int st_ = (expr);             \
    if (st_ != PHI_OK) return st_; \
  } while (0)

int validate(const phi_plan_desc& d, int64_t M) {
  if (M < 0 || M > 0x7fffffffLL) return PHI_ERR_ARG;
  if (d.image_n < 2 || d.image_n % 2) return PHI_ERR_ARG;
  if (!(d.oversample >= 1.0) || !(d.fov_rad > 0.0)) return PHI_ERR_ARG;
  double np = d.oversample * d.image_n;
  if (std::fabs(np - std::round(np)) > 1e-9 || static_cast<int64_t>(std::round(np)) % 2)
    return PHI_ERR_ARG;
  if (std::round(np) > 65536) return PHI_ERR_ARG;
  if (d.support < 2 || d.support % 2 || d.support > 64) return PHI_ERR_ARG;
  if (d.n_stacks < 1 || d.n_stacks > 126) return PHI_ERR_ARG;
  if (d.kmeans_max_iter < 1 || !(d.kmeans_tol >= 0.0)) return PHI_ERR_ARG;
  if (d.max_support < d.support || d.max_support > 256) return PHI_ERR_ARG;
  if (d.precision != PHI_F32 && d.precision != PHI_F64) return PHI_ERR_ARG;
  if (d.support_rule != PHI_SUPPORT_STACK && d.support_rule != PHI_SUPPORT_VIS) return PHI_ERR_ARG;
  if (!(d.alpha > 0.0) || !(d.quad_rel_tol > 0.0) || !(d.quad_abs_tol > 0.0)) return PHI_ERR_ARG;
  if (d.max_refine < 0 || d.max_refine > 8) return PHI_ERR_ARG;
  if (d.tile < 0 || d.tile > 4096) return PHI_ERR_ARG;
  if (d.kb_beta < 0.0 || d.cycles_per_panel < 0.0) return PHI_ERR_ARG;
  if (d.kernel_mode != PHI_KERNEL_QUADRATURE && d.kernel_mode != PHI_KERNEL_TABLE &&
      d.kernel_mode != PHI_KERNEL_RADIAL)
    return PHI_ERR_ARG;
  if (d.grid_staging < 0 || d.grid_staging > 2) return PHI_ERR_ARG;
  if (d.max_grid_mib < 0) return PHI_ERR_ARG;
  if (d.grid_deterministic != 0 && d.grid_deterministic != 1) return PHI_ERR_ARG;
  // uv-tile staging sums in shared memory with FP atomics first
  if (d.grid_deterministic && d.grid_staging == 1) return PHI_ERR_ARG;
  if (d.grid_staging && d.kernel_mode != PHI_KERNEL_TABLE) return PHI_ERR_ARG;
  if (d.kernel_mode == PHI_KERNEL_TABLE && !(d.table_tol > 0.0 && d.table_tol < 1.0))
    return PHI_ERR_ARG;
  return PHI_OK;
}

// Taps of every even support J <= jmax, each list sorted by distance of the
// tap (a, b) from the box centre (J/2 - 1/2, J/2 - 1/2), ties in raster order.
// A pure index permutation: it changes the order taps are visited in, never
// which taps are used.
int build_tap_order(Plan& p, int jmax, cudaStream_t s) {
  std::vector<int32_t> off;
  std::vector<uint16_t> codes;
  for (int J = 2; J <= jmax; J += 2) {
    off.push_back(static_cast<int32_t>(codes.size()));
    std::vector<std::pair<int, int>> taps;
    for (int b = 0; b < J; ++b)
      for (int a = 0; a < J; ++a) {
        const int da = 2 * a - (J - 1), db = 2 * b - (J - 1);
        taps.emplace_back(da * da + db * db, a | (b << 8));
      }
    std::stable_sort(taps.begin(), taps.end(),
                     [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
                       return x.first < y.first;
                     });
    for (const auto& t : taps) codes.push_back(static_cast<uint16_t>(t.second));
  }
  PHI_CUDA_TRY(owned_alloc(p, &p.tap_order, codes.size()));
  PHI_CUDA_TRY(owned_alloc(p, &p.tap_off, off.size()));
  PHI_CUDA_TRY(cudaMemcpyAsync(p.tap_order, codes.data(), codes.size() * sizeof(uint16_t),
                               cudaMemcpyHostToDevice, s));
  PHI_CUDA_TRY(cudaMemcpyAsync(p.tap_off, off.data(), off.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s));
  PHI_CUDA_TRY(cudaStreamSynchronize(s));
  return PHI_OK;
}

int build(Plan& p, const double* uvw, const double* weights, int64_t M, cudaStream_t s,
          const double* fixed_centres, const int32_t* fixed_jw) {
  const phi_plan_desc& d = p.d;
  p.N = d.image_n;
  p.npad = static_cast<int>(std::lround(d.oversample * d.image_n));
  p.K = d.n_stacks;
  p.M = M;
  p.dl = d.fov_rad / p.N;
  p.du = 1.0 / (p.npad * p.dl);
  p.R = 0.5 * d.alpha;
  p.beta = d.kb_beta > 0.0
               ? d.kb_beta
               : kPi * std::sqrt((double(d.support) / d.oversample) *
                                     (double(d.support) / d.oversample) *
                                     (d.oversample - 0.5) * (d.oversample - 0.5) -
                                 0.8);
  if (!(p.beta > 0.0)) return PHI_ERR_ARG;
  p.l_win = p.R / p.du;
  // Image corner and kernel window must stay below the horizon, and the
  // window must cover the image corners.
  const double half_fov = 0.5 * p.N * p.dl;
  if (p.l_win >= 1.0 || 2.0 * half_fov * half_fov >= 1.0) return PHI_ERR_HORIZON;
  if (std::sqrt(2.0) * half_fov > p.l_win) return PHI_ERR_ARG;
  p.n_win = std::sqrt(1.0 - p.l_win * p.l_win);
  p.c_support = p.l_win / (p.n_win * p.du);
  const double tol = std::min(d.quad_rel_tol, d.quad_abs_tol);
  // Gauss-Kronrod 15/31 panels of about 6 integrand cycles at the paper's
  // tolerance 1e-6, narrowing slowly with the tolerance (3.4 cycles at 1e-12):
  // the widths that gave the fewest tap-nodes, refinements included
  p.cycles_per_panel = d.cycles_per_panel > 0.0
                           ? d.cycles_per_panel
                           : std::min(8.0, std::max(1.0, 6.0 * std::pow(tol / 1e-6, 1.0 / 24.0)));

  int dev = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev));
  PHI_TRY(set_kernel_smem_limits());

  const int K = p.K;
  p.wbar.assign(K, 0.0);
  p.stack_off.assign(K + 1, 0);
  p.stack_jw.assign(K, 0);
  p.stack_maxabs.assign(K, 0.0);
  PHI_CUDA_TRY(owned_alloc(p, &p.counters, static_cast<size_t>(K) + 4));
  PHI_CUDA_TRY(cudaMemsetAsync(p.counters, 0, sizeof(unsigned long long) * (K + 4), s));

  Scratch tmp;
  const int nblk = std::max(1, std::min<int>(p.num_sms * 4,
                                             static_cast<int>((M + kPlanThreads - 1) / kPlanThreads)));
  double *w_fold = nullptr, *pmin = nullptr, *pmax = nullptr, *centres = nullptr,
         *upd = nullptr;
  unsigned long long* part = nullptr;
  int* kstate = nullptr;   // k-means: done flag, sweeps
  uint8_t* flag = nullptr;
  int32_t* stack = nullptr;
  PHI_CUDA_TRY(tmp.alloc(&w_fold, M));
  PHI_CUDA_TRY(tmp.alloc(&flag, M));
  PHI_CUDA_TRY(tmp.alloc(&stack, M));
  PHI_CUDA_TRY(tmp.alloc(&pmin, nblk));
  PHI_CUDA_TRY(tmp.alloc(&pmax, nblk));
  PHI_CUDA_TRY(tmp.alloc(&centres, K));
  PHI_CUDA_TRY(tmp.alloc(&part, static_cast<size_t>(nblk) * K * kAcc));
  PHI_CUDA_TRY(tmp.alloc(&kstate, 2));
  PHI_CUDA_TRY(tmp.alloc(&upd, 2 * K + 1));

  // --- fold and w range
  double wmin = 0.0, wmax = 0.0;
  if (M > 0) {
    unsigned long long* n_bad = p.counters + K + 2;   // free until the operator runs
    fold_kernel<<<nblk, kPlanThreads, 0, s>>>(uvw, M, d.conj_fold ? 1 : 0, w_fold, flag, pmin,
                                              pmax, n_bad);
    PHI_CUDA_TRY(cudaGetLastError());
    std::vector<double> hmin(nblk), hmax(nblk);
    unsigned long long hbad = 0;
    PHI_CUDA_TRY(cudaMemcpyAsync(hmin.data(), pmin, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaMemcpyAsync(hmax.data(), pmax, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaMemcpyAsync(&hbad, n_bad, sizeof(hbad), cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return PHI_ERR_ARG;
    PHI_CUDA_TRY(cudaMemsetAsync(n_bad, 0, sizeof(hbad), s));
    wmin = *std::min_element(hmin.begin(), hmin.end());
    wmax = *std::max_element(hmax.begin(), hmax.end());
  }

  // --- Algorithm 1 (or one nearest-centre assignment to given centres)
  std::vector<double> c(K);
  for (int q = 0; q < K; ++q)
    c[q] = fixed_centres ? fixed_centres[q]
                         : (K == 1) ? 0.5 * (wmin + wmax) : wmin + q * (wmax - wmin) / (K - 1);
  double eps = (wmax - wmin) / K;
  if (!(eps > 0.0)) eps = 1.0;
  PHI_CUDA_TRY(cudaMemcpyAsync(centres, c.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s));
  std::vector<double> hupd(2 * K + 1);
  p.kmeans_sweeps = 0;
  // fixed-point scale of the sums: |w| < 2^E for every w, so |w| 2^S < 2^62
  int E = 0;
  const double wabs = std::max(std::fabs(wmin), std::fabs(wmax));
  if (wabs > 0.0) std::frexp(wabs, &E);
  const int S = 62 - E;
  const int64_t chunk = ((M + nblk - 1) / nblk + 31) / 32 * 32;
  const size_t sweep_per_stack = (kPlanThreads / 32) * kAcc * sizeof(unsigned long long) +
                                 sizeof(double) + 2 * sizeof(float);
  const size_t sweep_smem = static_cast<size_t>(K) * sweep_per_stack;
  // The limit is a process-wide attribute of the function: a plan built at
  // the same time on another thread must not lower it under this launch, so
  // it is always set to what the most stacks a plan can have (126) need.
  PHI_CUDA_TRY(cudaFuncSetAttribute(kmeans_sweep_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(126 * sweep_per_stack)));
  if (M > 0 && fixed_centres) {
    kmeans_sweep_kernel<<<nblk, kPlanThreads, sweep_smem, s>>>(w_fold, M, chunk, centres, K, S,
                                                               stack, nullptr, nullptr);
    PHI_CUDA_TRY(cudaGetLastError());
    for (int q = 0; q < K; ++q) p.wbar[q] = c[q];
  } else if (M > 0) {
    // sweeps run in batches without a host round trip each: the update
    // kernel sets the done flag, after which the batch's remaining launches
    // return at once
    PHI_CUDA_TRY(cudaMemsetAsync(kstate, 0, 2 * sizeof(int), s));
    int hstate[2] = {0, 0};
    int launched = 0;
    while (!hstate[0] && launched < d.kmeans_max_iter) {
      const int batch = std::min(kSweepBatch, d.kmeans_max_iter - launched);
      for (int b = 0; b < batch; ++b) {
        kmeans_sweep_kernel<<<nblk, kPlanThreads, sweep_smem, s>>>(w_fold, M, chunk, centres, K,
                                                                   S, stack, part, kstate);
        kmeans_update_kernel<<<1, 32 * std::min(K, 32), sizeof(double) * K, s>>>(
            part, nblk, K, S, eps, d.kmeans_tol, d.kmeans_max_iter, centres, upd, kstate);
      }
      PHI_CUDA_TRY(cudaGetLastError());
      launched += batch;
      PHI_CUDA_TRY(cudaMemcpyAsync(hstate, kstate, sizeof(hstate), cudaMemcpyDeviceToHost, s));
      PHI_CUDA_TRY(cudaStreamSynchronize(s));
    }
    p.kmeans_sweeps = hstate[1];
    PHI_CUDA_TRY(cudaMemcpyAsync(hupd.data(), upd, sizeof(double) * (2 * K + 1),
                                 cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
    for (int q = 0; q < K; ++q) p.wbar[q] = hupd[q];
  } else {
    for (int q = 0; q < K; ++q) p.wbar[q] = c[q];
  }

  // --- classify: drop test, keys, per-stack max |dw| and kept counts
  const int tile = d.tile > 0 ? d.tile : 32;
  const int tiles_per_row = (p.npad + tile - 1) / tile;
  if (static_cast<int64_t>(tiles_per_row) * tiles_per_row >= (1 << 24)) return PHI_ERR_ARG;
  uint32_t *keys = nullptr, *vals = nullptr, *skeys = nullptr, *svals = nullptr;
  unsigned long long* stat = nullptr;  // [0..K) max |dw| bits, [K..2K) kept, [2K..3K) max jw
  PHI_CUDA_TRY(tmp.alloc(&keys, M));
  PHI_CUDA_TRY(tmp.alloc(&vals, M));
  PHI_CUDA_TRY(tmp.alloc(&skeys, M));
  PHI_CUDA_TRY(tmp.alloc(&svals, M));
  PHI_CUDA_TRY(tmp.alloc(&stat, 3 * static_cast<size_t>(K)));
  PHI_CUDA_TRY(cudaMemsetAsync(stat, 0, sizeof(unsigned long long) * 3 * K, s));
  std::vector<unsigned long long> hstat(3 * K, 0);
  if (M > 0) {
    classify_kernel<<<nblk, kPlanThreads, 0, s>>>(uvw, flag, w_fold, stack, centres, M, K, p.du,
                                                  p.npad, tile, tiles_per_row, keys, vals, stat,
                                                  stat + K);
    PHI_CUDA_TRY(cudaGetLastError());
    PHI_CUDA_TRY(cudaMemcpyAsync(hstat.data(), stat, sizeof(unsigned long long) * 2 * K,
                                 cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  p.n_kept = 0;
  for (int q = 0; q < K; ++q) {
    p.stack_off[q] = p.n_kept;
    p.n_kept += static_cast<int64_t>(hstat[K + q]);
    double maxabs;
    unsigned long long bits = hstat[q];
    std::memcpy(&maxabs, &bits, sizeof(double));
    p.stack_maxabs[q] = hstat[K + q] ? maxabs : 0.0;
    p.stack_jw[q] = hstat[K + q] ? d.support + 2 * static_cast<int32_t>(std::ceil(maxabs * p.c_support)) : 0;
    if (fixed_jw && hstat[K + q]) p.stack_jw[q] = fixed_jw[q];
  }
  p.stack_off[K] = p.n_kept;
  p.n_dropped = M - p.n_kept;
  // The per-visibility rule never exceeds the per-stack one, so checking the
  // per-stack value covers both.
  p.max_jw = 0;
  for (int q = 0; q < K; ++q) p.max_jw = std::max(p.max_jw, p.stack_jw[q]);
  if (p.max_jw > d.max_support) return PHI_ERR_SUPPORT;

  // --- sort by (stack, tile); dropped visibilities go last and are not kept
  if (M > 0) {
    size_t temp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, keys, skeys, vals, svals,
                                    static_cast<int>(M), 0, 32, s);
    void* temp = nullptr;
    PHI_CUDA_TRY(tmp.alloc(reinterpret_cast<unsigned char**>(&temp), temp_bytes));
    if (cub::DeviceRadixSort::SortPairs(temp, temp_bytes, keys, skeys, vals, svals,
                                        static_cast<int>(M), 0, 32, s) != cudaSuccess)
      return PHI_ERR_CUDA;
  }

  // --- records
  int32_t* d_stack_jw = nullptr;
  PHI_CUDA_TRY(tmp.alloc(&d_stack_jw, K));
  PHI_CUDA_TRY(cudaMemcpyAsync(d_stack_jw, p.stack_jw.data(), sizeof(int32_t) * K,
                               cudaMemcpyHostToDevice, s));
  const bool f64 = d.precision == PHI_F64;
  const size_t rec_bytes = f64 ? sizeof(VisRec<double>) : sizeof(VisRec<float>);
  PHI_CUDA_TRY(owned_alloc(p, reinterpret_cast<unsigned char**>(&p.recs), rec_bytes * p.n_kept));
  PHI_CUDA_TRY(owned_alloc(p, &p.perm, p.n_kept));
  const int per_vis = d.support_rule == PHI_SUPPORT_VIS ? 1 : 0;
  if (p.n_kept > 0) {
    if (f64)
      records_kernel<double><<<nblk, kPlanThreads, 0, s>>>(
          uvw, flag, w_fold, stack, centres, weights, svals, p.n_kept, p.du, d.support,
          p.c_support, per_vis, d_stack_jw, static_cast<VisRec<double>*>(p.recs), p.perm);
    else
      records_kernel<float><<<nblk, kPlanThreads, 0, s>>>(
          uvw, flag, w_fold, stack, centres, weights, svals, p.n_kept, p.du, d.support,
          p.c_support, per_vis, d_stack_jw, static_cast<VisRec<float>*>(p.recs), p.perm);
    PHI_CUDA_TRY(cudaGetLastError());
  }

  // --- table geometry (Sec. 5.1.1): sample spacing from the bilinear error
  // bound (half the budget per direction): h^2/8 times the second
  // derivative, bounded by (2 pi R)^2 in rho and (2 pi (1 - n_win))^2 in w
  if (d.kernel_mode == PHI_KERNEL_TABLE) {
    p.table_hr = std::sqrt(4.0 * d.table_tol) / (2.0 * kPi * p.R);
    p.table_hw = std::sqrt(4.0 * d.table_tol) / (2.0 * kPi * (1.0 - p.n_win));
    double dmax = 0.0;
    for (int q = 0; q < K; ++q) dmax = std::max(dmax, p.stack_maxabs[q]);
    const double rmax = std::sqrt(2.0) * std::max(p.max_jw, d.support) / 2.0 + 2.0;
    p.table_nr = static_cast<int64_t>(std::ceil(rmax / p.table_hr)) + 2;
    p.table_nw = static_cast<int64_t>(std::ceil(dmax / p.table_hw)) + 2;
    if (p.table_nr * p.table_nw > (int64_t(1) << 31) || p.table_nw - 2 >= (1 << 24))
      return PHI_ERR_ARG;
  }

  // --- stack groups: the stacks with visibilities, `group` at a time, their
  // grids resident together (as many as fit max_grid_mib, at least one)
  const size_t grid_bytes = 2 * (f64 ? sizeof(double) : sizeof(float)) *
                            static_cast<size_t>(p.npad) * p.npad;
  // a deterministic plan also holds two int64 per cell of every resident grid
  const size_t fx_bytes =
      d.grid_deterministic ? 2 * sizeof(long long) * static_cast<size_t>(p.npad) * p.npad : 0;
  p.group_stacks.clear();
  for (int q = 0; q < K; ++q)
    if (p.stack_off[q + 1] > p.stack_off[q]) p.group_stacks.push_back(q);
  const double budget = (d.max_grid_mib > 0 ? d.max_grid_mib : 4096) * 1048576.0;
  p.group = static_cast<int>(std::max<double>(1.0, std::floor(budget / (grid_bytes + fx_bytes))));
  p.group = std::max(1, std::min<int>(p.group, static_cast<int>(p.group_stacks.size())));
  p.group_off.assign(1, 0);
  for (size_t g = 0; g < p.group_stacks.size(); g += p.group)
    p.group_off.push_back(static_cast<int64_t>(std::min(p.group_stacks.size(), g + p.group)));
  std::vector<int32_t> slot(K, 0);
  for (size_t g = 0; g + 1 < p.group_off.size(); ++g)
    for (int64_t i = p.group_off[g]; i < p.group_off[g + 1]; ++i)
      slot[p.group_stacks[i]] = static_cast<int32_t>(i - p.group_off[g]);

  // --- work items of the table path's staged kernels: runs of equal key in
  // the sorted kept records (grid_staging 1: uv tiles, in record order;
  // grid_staging 2: w-rows, through the index p.row_idx), split into items of
  // at most max_records records
  p.tile = tile;
  p.tiles_per_row = tiles_per_row;
  p.stack_item_off.assign(K + 1, 0);
  p.stack_staged.assign(K, 0);
  if (d.kernel_mode == PHI_KERNEL_TABLE && d.grid_staging && p.n_kept > 0) {
    const int64_t n = p.n_kept;
    const uint32_t* ikeys = skeys;   // uv-tile keys of the kept records, in order
    int max_records = kItemRecords;
    if (d.grid_staging == 2) {
      uint32_t *rk = nullptr, *rv = nullptr, *rks = nullptr;
      PHI_CUDA_TRY(tmp.alloc(&rk, n));
      PHI_CUDA_TRY(tmp.alloc(&rv, n));
      PHI_CUDA_TRY(tmp.alloc(&rks, n));
      PHI_CUDA_TRY(owned_alloc(p, &p.row_idx, n));
      const int last_row = static_cast<int>(p.table_nw - 2);
      if (f64)
        row_key_kernel<double><<<nblk, kPlanThreads, 0, s>>>(
            static_cast<const VisRec<double>*>(p.recs), n, 1.0 / p.table_hw, last_row, rk, rv);
      else
        row_key_kernel<float><<<nblk, kPlanThreads, 0, s>>>(
            static_cast<const VisRec<float>*>(p.recs), n, static_cast<float>(1.0 / p.table_hw),
            last_row, rk, rv);
      PHI_CUDA_TRY(cudaGetLastError());
      size_t bytes = 0;
      cub::DeviceRadixSort::SortPairs(nullptr, bytes, rk, rks, rv, p.row_idx,
                                      static_cast<int>(n), 0, 32, s);
      void* sort_tmp = nullptr;
      PHI_CUDA_TRY(tmp.alloc(reinterpret_cast<unsigned char**>(&sort_tmp), bytes));
      if (cub::DeviceRadixSort::SortPairs(sort_tmp, bytes, rk, rks, rv, p.row_idx,
                                          static_cast<int>(n), 0, 32, s) != cudaSuccess)
        return PHI_ERR_CUDA;
      ikeys = rks;
      max_records = kRowItemRecords;
    }
    uint32_t *flag = nullptr, *pos = nullptr, *tkey = nullptr;
    int32_t* tstart = nullptr;
    PHI_CUDA_TRY(tmp.alloc(&flag, n));
    PHI_CUDA_TRY(tmp.alloc(&pos, n));
    PHI_CUDA_TRY(tmp.alloc(&tkey, n));
    PHI_CUDA_TRY(tmp.alloc(&tstart, n));
    tile_flag_kernel<<<nblk, kPlanThreads, 0, s>>>(ikeys, n, flag);
    PHI_CUDA_TRY(cudaGetLastError());
    size_t scan_bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, flag, pos, static_cast<int>(n), s);
    void* scan_tmp = nullptr;
    PHI_CUDA_TRY(tmp.alloc(reinterpret_cast<unsigned char**>(&scan_tmp), scan_bytes));
    if (cub::DeviceScan::ExclusiveSum(scan_tmp, scan_bytes, flag, pos, static_cast<int>(n), s) !=
        cudaSuccess)
      return PHI_ERR_CUDA;
    tile_scatter_kernel<<<nblk, kPlanThreads, 0, s>>>(ikeys, flag, pos, n, tstart, tkey);
    PHI_CUDA_TRY(cudaGetLastError());
    uint32_t last[2] = {0, 0};
    PHI_CUDA_TRY(cudaMemcpyAsync(&last[0], pos + n - 1, 4, cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaMemcpyAsync(&last[1], flag + n - 1, 4, cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t n_runs = static_cast<int64_t>(last[0]) + last[1];
    std::vector<int32_t> hstart(n_runs + 1);
    std::vector<uint32_t> hkey(n_runs);
    PHI_CUDA_TRY(cudaMemcpyAsync(hstart.data(), tstart, 4 * n_runs, cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaMemcpyAsync(hkey.data(), tkey, 4 * n_runs, cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
    hstart[n_runs] = static_cast<int32_t>(n);
    // items: start and end interleaved, item_start[2 i] = start, [2 i + 1] = end
    std::vector<int32_t> se;
    std::vector<uint32_t> ikey;
    int cur_stack = -1;
    for (int64_t t = 0; t < n_runs; ++t) {
      const int st = static_cast<int>(hkey[t] >> 24);
      while (cur_stack < st) p.stack_item_off[++cur_stack] = static_cast<int64_t>(ikey.size());
      for (int32_t r = hstart[t]; r < hstart[t + 1]; r += max_records) {
        se.push_back(r);
        se.push_back(std::min<int32_t>(r + max_records, hstart[t + 1]));
        ikey.push_back(hkey[t]);
      }
    }
    while (cur_stack < K) p.stack_item_off[++cur_stack] = static_cast<int64_t>(ikey.size());
    for (int q = 0; q < K; ++q) p.stack_staged[q] = 1;
    PHI_CUDA_TRY(owned_alloc(p, &p.item_start, se.size()));
    PHI_CUDA_TRY(owned_alloc(p, &p.item_key, ikey.size()));
    PHI_CUDA_TRY(cudaMemcpyAsync(p.item_start, se.data(), 4 * se.size(), cudaMemcpyHostToDevice, s));
    PHI_CUDA_TRY(cudaMemcpyAsync(p.item_key, ikey.data(), 4 * ikey.size(), cudaMemcpyHostToDevice, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
  }

  // --- tables, grid, FFT plan
  const size_t tsize = f64 ? sizeof(double) : sizeof(float);
  const int64_t nodes = panel_table_offset(kMaxPanels + 1);
  PHI_CUDA_TRY(owned_alloc(p, &p.node_omn, nodes));
  PHI_CUDA_TRY(owned_alloc(p, reinterpret_cast<unsigned char**>(&p.node_hk), tsize * nodes));
  PHI_CUDA_TRY(owned_alloc(p, reinterpret_cast<unsigned char**>(&p.node_hd), tsize * nodes));
  PHI_TRY(build_tap_order(p, std::max(p.max_jw, 2), s));
  PHI_CUDA_TRY(owned_alloc(p, &p.omn_pix, static_cast<size_t>(p.N) * p.N));
  PHI_CUDA_TRY(owned_alloc(p, reinterpret_cast<unsigned char**>(&p.corr_pix),
                           tsize * p.N * static_cast<size_t>(p.N)));
  PHI_CUDA_TRY(owned_alloc(p, &p.group_stacks_dev, std::max<size_t>(1, p.group_stacks.size())));
  PHI_CUDA_TRY(owned_alloc(p, &p.stack_slot_dev, K));
  PHI_CUDA_TRY(owned_alloc(p, &p.wbar_dev, K));
  if (!p.group_stacks.empty())
    PHI_CUDA_TRY(cudaMemcpyAsync(p.group_stacks_dev, p.group_stacks.data(),
                                 4 * p.group_stacks.size(), cudaMemcpyHostToDevice, s));
  PHI_CUDA_TRY(cudaMemcpyAsync(p.stack_slot_dev, slot.data(), 4 * K, cudaMemcpyHostToDevice, s));
  PHI_CUDA_TRY(cudaMemcpyAsync(p.wbar_dev, p.wbar.data(), 8 * K, cudaMemcpyHostToDevice, s));
  PHI_CUDA_TRY(owned_alloc(p, reinterpret_cast<unsigned char**>(&p.grid),
                           grid_bytes * static_cast<size_t>(p.group)));
  PHI_TRY(launch_node_tables(p, s));
  PHI_TRY(launch_pixel_tables(p, s));
  if (d.grid_deterministic) {
    PHI_CUDA_TRY(owned_alloc(p, &p.fx_cells, 2 * static_cast<size_t>(p.npad) * p.npad * p.group));
    PHI_CUDA_TRY(owned_alloc(p, &p.fx_max, 1));
    PHI_CUDA_TRY(owned_alloc(p, &p.fx_exp, 2));
    double* bound = nullptr;
    PHI_CUDA_TRY(tmp.alloc(&bound, kMaxPanels));
    PHI_TRY(compute_kernel_bound(p, bound, s));
  }
  if (d.kernel_mode == PHI_KERNEL_TABLE) {
    const size_t pair = 2 * 2 * tsize;
    PHI_CUDA_TRY(owned_alloc(p, reinterpret_cast<unsigned char**>(&p.table),
                             pair * (p.table_nw - 1) * p.table_nr));
    PHI_TRY(build_kernel_table(p, s));
  }
  if (d.kernel_mode == PHI_KERNEL_RADIAL) PHI_TRY(build_radial_tables(p, s));
  if (cufftCreate(&p.fft) != CUFFT_SUCCESS) return PHI_ERR_CUDA;
  p.fft_ok = true;
  size_t work = 0;
  if (cufftMakePlan2d(p.fft, p.npad, p.npad, f64 ? CUFFT_Z2Z : CUFFT_C2C, &work) != CUFFT_SUCCESS)
    return PHI_ERR_OOM;
  p.device_bytes += static_cast<int64_t>(work);
  if (p.group > 1) {
    if (cufftCreate(&p.fft_batch) != CUFFT_SUCCESS) return PHI_ERR_CUDA;
    p.fft_batch_ok = true;
    int dims[2] = {p.npad, p.npad};
    const int dist = p.npad * p.npad;
    size_t work_b = 0;
    if (cufftMakePlanMany(p.fft_batch, 2, dims, nullptr, 1, dist, nullptr, 1, dist,
                          f64 ? CUFFT_Z2Z : CUFFT_C2C, p.group, &work_b) != CUFFT_SUCCESS)
      return PHI_ERR_OOM;
    p.device_bytes += static_cast<int64_t>(work_b);
  }
  PHI_CUDA_TRY(cudaStreamSynchronize(s));
  return PHI_OK;
}

}  // namespace
}  // namespace phi

extern "C" int phi_plan_desc_default(phi_plan_desc* d) {
  if (!d) return PHI_ERR_ARG;
  std::memset(d, 0, sizeof(*d));
  d->support = 4;
  d->n_stacks = 1;
  d->kmeans_max_iter = 100;
  d->conj_fold = 0;
  d->max_support = 64;
  d->precision = PHI_F32;
  d->support_rule = PHI_SUPPORT_STACK;
  d->max_refine = 3;
  d->tile = 32;
  d->oversample = 2.0;
  d->kmeans_tol = 1e-3;
  d->alpha = 1.0;
  d->quad_rel_tol = 1e-6;
  d->quad_abs_tol = 1e-6;
  d->kb_beta = 0.0;
  d->cycles_per_panel = 0.0;
  d->kernel_mode = PHI_KERNEL_QUADRATURE;
  d->grid_staging = 0;
  d->table_tol = 1e-4;
  return PHI_OK;
}

namespace {

int create(phi_plan_t* out, const phi_plan_desc* desc, const double* uvw_dev,
           const double* weights_dev, int64_t n_vis, const double* centres,
           const int32_t* stack_jw, void* stream) {
  if (!out || !desc) return PHI_ERR_ARG;
  *out = nullptr;
  int st = phi::validate(*desc, n_vis);
  if (st != PHI_OK) return st;
  if (n_vis > 0 && !uvw_dev) return PHI_ERR_ARG;
  if (centres) {
    for (int q = 0; q < desc->n_stacks; ++q)
      if (!std::isfinite(centres[q])) return PHI_ERR_ARG;
  }
  if (stack_jw) {
    if (!centres || desc->support_rule != PHI_SUPPORT_STACK) return PHI_ERR_ARG;
    for (int q = 0; q < desc->n_stacks; ++q)
      if (stack_jw[q] < 2 || stack_jw[q] % 2 || stack_jw[q] > desc->max_support) return PHI_ERR_ARG;
  }
  phi_plan* p = new (std::nothrow) phi_plan();
  if (!p) return PHI_ERR_OOM;
  p->d = *desc;
  st = phi::build(*p, uvw_dev, weights_dev, n_vis, static_cast<cudaStream_t>(stream), centres,
                  stack_jw);
  if (st != PHI_OK) {
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    phi::free_plan(p);
    delete p;
    return st;
  }
  *out = p;
  return PHI_OK;
}

}  // namespace

extern "C" int phi_plan_create(phi_plan_t* out, const phi_plan_desc* desc, const double* uvw_dev,
                               const double* weights_dev, int64_t n_vis, void* stream) {
  return create(out, desc, uvw_dev, weights_dev, n_vis, nullptr, nullptr, stream);
}

extern "C" int phi_plan_create_fixed(phi_plan_t* out, const phi_plan_desc* desc,
                                     const double* uvw_dev, const double* weights_dev,
                                     int64_t n_vis, const double* centres,
                                     const int32_t* stack_jw, void* stream) {
  if (!centres) return PHI_ERR_ARG;
  return create(out, desc, uvw_dev, weights_dev, n_vis, centres, stack_jw, stream);
}

extern "C" void phi_plan_destroy(phi_plan_t plan) {
  if (!plan) return;
  phi::free_plan(plan);
  delete plan;
}

extern "C" int phi_plan_info(phi_plan_t plan, phi_plan_summary* info, double* wbar, int64_t* counts,
                             int32_t* jw) {
  if (!plan) return PHI_ERR_ARG;
  const phi::Plan& p = *plan;
  if (info) {
    info->n_vis = p.M;
    info->n_kept = p.n_kept;
    info->n_dropped = p.n_dropped;
    info->device_bytes = p.device_bytes;
    info->image_n = p.N;
    info->npad = p.npad;
    info->n_stacks = p.K;
    info->kmeans_sweeps = p.kmeans_sweeps;
    info->max_jw = p.max_jw;
    info->precision = p.d.precision;
    info->du = p.du;
    info->dl = p.dl;
    info->beta = p.beta;
    info->window_radius = p.R;
    info->support_coeff = p.c_support;
    info->kernel_mode = p.d.kernel_mode;
    info->group = p.group;
    info->table_n_rho = p.table_nr;
    info->table_n_w = p.table_nw;
    info->table_h_rho = p.table_hr;
    info->table_h_w = p.table_hw;
  }
  for (int q = 0; q < p.K; ++q) {
    if (wbar) wbar[q] = p.wbar[q];
    if (counts) counts[q] = p.stack_off[q + 1] - p.stack_off[q];
    if (jw) jw[q] = p.stack_jw[q];
  }
  return PHI_OK;
}

extern "C" int phi_plan_stats(phi_plan_t plan, int64_t* n_unconverged, int64_t* n_taps,
                              int64_t* n_tap_nodes, int reset, void* stream) {
  if (!plan) return PHI_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long h[4] = {0, 0, 0, 0};
  PHI_CUDA_TRY(cudaMemcpyAsync(h, plan->counters + plan->K, sizeof(h), cudaMemcpyDeviceToHost, s));
  PHI_CUDA_TRY(cudaStreamSynchronize(s));
  if (n_unconverged) *n_unconverged = static_cast<int64_t>(h[0]);
  if (n_taps) *n_taps = static_cast<int64_t>(h[1]);
  if (n_tap_nodes) *n_tap_nodes = static_cast<int64_t>(h[3]);
  if (reset) {
    PHI_CUDA_TRY(cudaMemsetAsync(plan->counters + plan->K, 0, 4 * sizeof(unsigned long long), s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return PHI_OK;
}

extern "C" const char* phi_error_string(int status) {
  switch (status) {
    case PHI_OK: return "ok";
    case PHI_ERR_ARG: return "invalid argument";
    case PHI_ERR_OOM: return "device out of memory";
    case PHI_ERR_CUDA: return "CUDA or cuFFT call failed";
    case PHI_ERR_HORIZON: return "image or kernel window reaches the horizon";
    case PHI_ERR_SUPPORT: return "w-projection support exceeds max_support";
    case PHI_ERR_TIMEOUT: return "bounded wait timed out";
    case PHI_ERR_STATE: return "call does not apply to this plan";
    default: return "unknown status";
  }
}
