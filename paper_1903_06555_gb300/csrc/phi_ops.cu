// Hot-path kernels of the w-stacking w-projection operator on GB300 (sm_103a):
//
//   prep    S~_k and Z (Eq. S~_k): padded grid <- x e^{2 pi i wbar_k (1-n)} / (g n)
//   F       cuFFT, unnormalised, in place
//   degrid  fused [GC] quadrature (Eq. analytic_convolution_hankel) + G + W + fold
//   grid    fused [GC] quadrature + G^H (Eq. stacked adjoint) with float atomics
//   finish  F^H output -> crop (Z^T) -> conj(S~_k) -> real part -> sum over stacks
//
// Kernel evaluation.  One warp owns one visibility.  The chirp part of the
// integrand, h(r_j) = 2 pi h_p g(r_j) r_j e^{-2 pi i dw (n(r_j) - 1)}, is the
// same for all J_w^2 taps of the visibility, so the lanes first build it at
// the Gauss-Kronrod 15/31 nodes of an a-priori partition of [0, R] into
// equal panels (FP64 phase argument, tabulated 1 - n(r_j) and g(r_j)), then
// each lane takes one tap and sums J0(2 pi rho r_j) h(r_j) with the Kronrod
// weights, and, per panel, the difference against the embedded Gauss rule
// as the error estimate (FP32 path: in paired f32x2 arithmetic, two nodes
// per instruction).  A chunk of 32 taps whose estimate misses
// max(abs_tol, rel_tol |K|) is recomputed with twice the panels (up to
// max_refine times); taps still above tolerance are counted.  The degridder
// and the gridder run this identical routine, so [GC] and its conjugate
// transpose pair exactly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "bessel_j0.cuh"
#include "table_index.cuh"
#include "fixed_point.cuh"
#include "phi_internal.cuh"

namespace phi {

// ---------------------------------------------------------------------------
// Gauss-Kronrod 15/31 rule on [-1, 1]: the 15-point Gauss-Legendre rule and
// its Kronrod extension (the zeros of the Stieltjes polynomial E_16), as
// computed by gk_rule.py in this directory from the rule's definition.
// Node j = 0..30 runs from -1 to 1; i = 0..15 indexes |x| from the outermost
// node to the centre.  The Gauss nodes are the odd j (i odd, and the centre).
// ---------------------------------------------------------------------------
constexpr int kNodes = kNodesPerPanel;   // 31
__host__ __device__ constexpr double gk_abs_node(int i) {
  return i == 0 ? 0.998002298693397060285172840152271209
       : i == 1 ? 0.987992518020485428489565718586612581
       : i == 2 ? 0.967739075679139134257347978784337225
       : i == 3 ? 0.937273392400705904307758947710209471
       : i == 4 ? 0.897264532344081900882509656454495883
       : i == 5 ? 0.848206583410427216200648320774216851
       : i == 6 ? 0.790418501442465932967649294817947347
       : i == 7 ? 0.72441773136017004741618605461393801
       : i == 8 ? 0.650996741297416970533735895313274693
       : i == 9 ? 0.570972172608538847537226737253910641
       : i == 10 ? 0.485081863640239680693655740232350613
       : i == 11 ? 0.394151347077563369897207370981045468
       : i == 12 ? 0.299180007153168812166780024266388963
       : i == 13 ? 0.201194093997434522300628303394596208
       : i == 14 ? 0.101142066918717499027074231447392339
       : i == 15 ? 0.0
                : 0.0;
}
__host__ __device__ constexpr double gk_kronrod_weight(int i) {
  return i == 0 ? 0.00537747987292334898779205143012764982
       : i == 1 ? 0.0150079473293161225383747630758072681
       : i == 2 ? 0.0254608473267153201868740010196533594
       : i == 3 ? 0.0353463607913758462220379484783600481
       : i == 4 ? 0.0445897513247648766082272993732796902
       : i == 5 ? 0.0534815246909280872653431472394302968
       : i == 6 ? 0.0620095678006706402851392309608029322
       : i == 7 ? 0.0698541213187282587095200770991474758
       : i == 8 ? 0.0768496807577203788944327774826590067
       : i == 9 ? 0.0830805028231330210382892472861037896
       : i == 10 ? 0.0885644430562117706472754436937743032
       : i == 11 ? 0.0931265981708253212254868727473457186
       : i == 12 ? 0.0966427269836236785051799076275893351
       : i == 13 ? 0.0991735987217919593323931734846031311
       : i == 14 ? 0.100769845523875595044946662617569722
       : i == 15 ? 0.101330007014791549017374792767492547
                : 0.0;
}
__host__ __device__ constexpr double gk_gauss_weight(int i) {  // at gk_abs_node(i), 0 for Kronrod-only
  return i == 1 ? 0.0307532419961172683546283935772044177
       : i == 3 ? 0.0703660474881081247092674164506673385
       : i == 5 ? 0.107159220467171935011869546685869303
       : i == 7 ? 0.139570677926154314447804794511028323
       : i == 9 ? 0.166269205816993933553200860481208811
       : i == 11 ? 0.186161000015562211026800561866422825
       : i == 13 ? 0.198431485327111576456118326443839325
       : i == 15 ? 0.202578241925561272880620199967519315
                : 0.0;
}
__host__ __device__ constexpr int gk_fold(int j) { return j < 15 ? j : 30 - j; }
__host__ __device__ constexpr double gk_node(int j) {
  return j < 15 ? -gk_abs_node(j) : gk_abs_node(30 - j);
}
__host__ __device__ constexpr double gk_wk(int j) { return gk_kronrod_weight(gk_fold(j)); }
__host__ __device__ constexpr double gk_wd(int j) {  // Kronrod minus Gauss weight
  return gk_kronrod_weight(gk_fold(j)) - gk_gauss_weight(gk_fold(j));
}
__host__ __device__ constexpr double gk_gw(int j) {  // Gauss weight (0: Kronrod-only node)
  return gk_gauss_weight(gk_fold(j));
}

// Nodes in the precision of the integrand, read uniformly by the whole warp.
__constant__ float c_gk_node_f[kNodes] = {
    -0.99800229869339707f, -0.98799251802048538f, -0.96773907567913908f, -0.93727339240070595f,
    -0.89726453234408188f, -0.84820658341042721f, -0.79041850144246595f, -0.72441773136017007f,
    -0.65099674129741703f, -0.57097217260853883f, -0.4850818636402397f, -0.39415134707756339f,
    -0.29918000715316884f, -0.20119409399743451f, -0.10114206691871749f, 0.0f,
    0.10114206691871749f, 0.20119409399743451f, 0.29918000715316884f, 0.39415134707756339f,
    0.4850818636402397f, 0.57097217260853883f, 0.65099674129741703f, 0.72441773136017007f,
    0.79041850144246595f, 0.84820658341042721f, 0.89726453234408188f, 0.93727339240070595f,
    0.96773907567913908f, 0.98799251802048538f, 0.99800229869339707f};
__constant__ double c_gk_node_d[kNodes] = {
    -0.998002298693397060285172840152271209, -0.987992518020485428489565718586612581,
    -0.967739075679139134257347978784337225, -0.937273392400705904307758947710209471,
    -0.897264532344081900882509656454495883, -0.848206583410427216200648320774216851,
    -0.790418501442465932967649294817947347, -0.72441773136017004741618605461393801,
    -0.650996741297416970533735895313274693, -0.570972172608538847537226737253910641,
    -0.485081863640239680693655740232350613, -0.394151347077563369897207370981045468,
    -0.299180007153168812166780024266388963, -0.201194093997434522300628303394596208,
    -0.101142066918717499027074231447392339, 0.0,
    0.101142066918717499027074231447392339, 0.201194093997434522300628303394596208,
    0.299180007153168812166780024266388963, 0.394151347077563369897207370981045468,
    0.485081863640239680693655740232350613, 0.570972172608538847537226737253910641,
    0.650996741297416970533735895313274693, 0.72441773136017004741618605461393801,
    0.790418501442465932967649294817947347, 0.848206583410427216200648320774216851,
    0.897264532344081900882509656454495883, 0.937273392400705904307758947710209471,
    0.967739075679139134257347978784337225, 0.987992518020485428489565718586612581,
    0.998002298693397060285172840152271209};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
// J0(pi u): the FP32 path uses the compact approximation of bessel_j0.cuh,
// the FP64 path CUDA's j0.
__device__ __forceinline__ float j0_hc(float u) { return j0_halfcycles(u); }
__device__ __forceinline__ double j0_hc(double u) { return j0(kPi * u); }
__device__ __forceinline__ float j0_hc_large(float u) { return j0_large(u); }
__device__ __forceinline__ double j0_hc_large(double u) { return j0(kPi * u); }
// Warp vote: every active lane's lowest node argument lies past the
// small-argument formula (u > kJ0Split strictly, as j0_halfcycles tests).
// Node arguments exceed a - Bh by at least (1 - 0.9915) Bh, far more than the
// rounding of a - Bh, so the vote never sends a node to the wrong formula.
// FP64 has a single formula.
__device__ __forceinline__ bool panel_all_large(float lo, bool active) {
  return __all_sync(0xffffffffu, !active || lo > kJ0Split);
}
__device__ __forceinline__ bool panel_all_large(double, bool) { return false; }
__device__ __forceinline__ float gk_node_c(float, int j) { return c_gk_node_f[j]; }
__device__ __forceinline__ double gk_node_c(double, int j) { return c_gk_node_d[j]; }
// Square root for error estimates and tolerance tests only: the hardware
// approximation in FP32 (relative error ~2^-22), the correctly rounded one in FP64.
__device__ __forceinline__ float est_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double est_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ void sincos_pi(float a, float* s, float* c) { sincospif(a, s, c); }
__device__ __forceinline__ void sincos_pi(double a, double* s, double* c) { sincospi(a, s, c); }

template <typename C> __device__ __forceinline__ C cmake(double x, double y);
template <> __device__ __forceinline__ float2 cmake<float2>(double x, double y) {
  return make_float2(static_cast<float>(x), static_cast<float>(y));
}
template <> __device__ __forceinline__ double2 cmake<double2>(double x, double y) {
  return make_double2(x, y);
}

__device__ __forceinline__ void atomic_add_c(float2* p, float2 v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_c(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// The fixed-point target shifted by `off` cells, as a grid pointer is.
__device__ __forceinline__ FixedGrid fixed_offset(const FixedGrid& fx, int64_t off) {
  FixedGrid r;
  r.cells = fx.cells ? fx.cells + 2 * off : nullptr;
  r.exp = fx.exp;
  return r;
}

// Adds a gridding contribution to cell gi: to the complex grid with FP
// atomics, or, for a deterministic plan, to the cell's fixed-point pair.
template <typename C>
__device__ __forceinline__ void grid_add(C* grid_out, const FixedGrid& fx, int64_t gi,
                                         const C& add) {
  if (fx.cells) {
    const int e = __ldg(fx.exp);
    atomicAdd(fx.cells + 2 * gi, static_cast<unsigned long long>(fixed_point(add.x, e)));
    atomicAdd(fx.cells + 2 * gi + 1, static_cast<unsigned long long>(fixed_point(add.y, e)));
  } else {
    atomic_add_c(grid_out + gi, add);
  }
}

// Circular grid index q mod n outside the loops: a division by a run-time n
// (its int <-> float conversions run on the FP64 unit, about 1/64 of the FP32
// rate here).  Not inlined, so that its call can be skipped by a branch
// rather than if-converted into every tap.
__device__ __noinline__ int wrap_index_mod(int q, int n) {
  q %= n;
  return q < 0 ? q + n : q;
}

// Circular grid index q mod n in 32-bit arithmetic.  The records hold
// centred cell indices (the box of a kept visibility lies within
// [-n/2 - J_w/2, n/2 + J_w/2]), so one conditional add or subtract of n
// wraps every tap; anything farther out takes the division.
__device__ __forceinline__ int wrap_index(int q, int n) {
  if (q < 0) q += n;
  if (q >= n) q -= n;
  if (static_cast<unsigned>(q) >= static_cast<unsigned>(n)) q = wrap_index_mod(q, n);
  return q;
}

// 2-D transform of the radial Kaiser-Bessel kernel (support J = 2a, shape
// beta): g(r) = 2 pi a^2 I1(z) / (z I0(beta)), z^2 = beta^2 - (2 pi a r)^2,
// with J1(|z|)/|z| in place of I1(z)/z where z^2 < 0 (Lewitt 1990).
__device__ double taper_g(double r, double a, double beta, double i0beta) {
  double q = 2.0 * kPi * a * r;
  double z2 = beta * beta - q * q;
  double f;
  if (fabs(z2) < 1e-12) {
    f = 0.5 + z2 / 16.0;
  } else if (z2 > 0.0) {
    double z = sqrt(z2);
    f = cyl_bessel_i1(z) / z;
  } else {
    double z = sqrt(-z2);
    f = j1(z) / z;
  }
  return 2.0 * kPi * a * a * f / i0beta;
}

// ---------------------------------------------------------------------------
// Tables built once per plan
// ---------------------------------------------------------------------------
template <typename T>
__global__ void node_table_kernel(double R, double du, double a, double beta, double* omn,
                                  T* hk, T* hd, int64_t total) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= total) return;
  int npan = 1;
  while (npan < kMaxPanels && panel_table_offset(npan + 1) <= j) ++npan;
  const int64_t off = panel_table_offset(npan);
  int64_t local = j - off;
  int p = static_cast<int>(local / kNodes);
  int k = static_cast<int>(local % kNodes);
  double hw = R / (2.0 * npan);
  double r = hw * (2.0 * p + 1.0 + gk_node(k));
  double l = r / du;
  double s = l * l;
  omn[j] = s / (1.0 + sqrt(1.0 - s));
  double h = 2.0 * kPi * hw * taper_g(r, a, beta, cyl_bessel_i0(beta)) * r;
  hk[j] = static_cast<T>(gk_wk(k) * h);
  // FP32 quadrature forms its estimate from panel sums with the Gauss weight
  // (zero at Kronrod-only nodes), FP64 from the Kronrod-minus-Gauss weight
  hd[j] = static_cast<T>((sizeof(T) == 4 ? gk_gw(k) : gk_wd(k)) * h);
}

template <typename T>
__global__ void pixel_table_kernel(int N, double dl, double du, double a, double beta,
                                   double* omn, T* corr) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)N * N) return;
  int row = static_cast<int>(idx / N), col = static_cast<int>(idx % N);
  double l = (col - N / 2) * dl, m = (row - N / 2) * dl;
  double s = l * l + m * m;
  double n = sqrt(1.0 - s);
  omn[idx] = s / (1.0 + n);
  double g = taper_g(du * sqrt(s), a, beta, cyl_bessel_i0(beta));
  corr[idx] = static_cast<T>(1.0 / (g * n));
}

int launch_node_tables(Plan& p, cudaStream_t s) {
  int64_t total = panel_table_offset(kMaxPanels + 1);
  int blocks = static_cast<int>((total + 255) / 256);
  double a = 0.5 * p.d.support;
  if (p.d.precision == PHI_F64)
    node_table_kernel<double><<<blocks, 256, 0, s>>>(p.R, p.du, a, p.beta, p.node_omn,
                                                    static_cast<double*>(p.node_hk),
                                                    static_cast<double*>(p.node_hd), total);
  else
    node_table_kernel<float><<<blocks, 256, 0, s>>>(p.R, p.du, a, p.beta, p.node_omn,
                                                   static_cast<float*>(p.node_hk),
                                                   static_cast<float*>(p.node_hd), total);
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}

int launch_pixel_tables(Plan& p, cudaStream_t s) {
  int64_t total = (int64_t)p.N * p.N;
  int blocks = static_cast<int>((total + 255) / 256);
  double a = 0.5 * p.d.support;
  if (p.d.precision == PHI_F64)
    pixel_table_kernel<double><<<blocks, 256, 0, s>>>(p.N, p.dl, p.du, a, p.beta, p.omn_pix,
                                                     static_cast<double*>(p.corr_pix));
  else
    pixel_table_kernel<float><<<blocks, 256, 0, s>>>(p.N, p.dl, p.du, a, p.beta, p.omn_pix,
                                                    static_cast<float*>(p.corr_pix));
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}

// ---------------------------------------------------------------------------
// Image-domain steps
// ---------------------------------------------------------------------------

// S~_k then Z for every stack of a group (blockIdx.y = slot): grid cell
// (qv, qu) holds padded pixel P = (q + Npad/2) mod Npad (the centred image
// moved to index 0), i.e. image pixel P - (Npad - N)/2, or zero outside.
template <typename T, typename C>
__global__ void prep_kernel(const T* __restrict__ x, const double* __restrict__ omn,
                            const T* __restrict__ corr, int N, int npad,
                            const double* __restrict__ wbar, const int32_t* __restrict__ stacks,
                            C* __restrict__ grids) {
  const int off = (npad - N) / 2;
  const double wb = wbar[stacks[blockIdx.y]];
  C* grid = grids + static_cast<int64_t>(blockIdx.y) * npad * npad;
  for (int qv = blockIdx.x; qv < npad; qv += gridDim.x) {
    int pv = qv + npad / 2;
    if (pv >= npad) pv -= npad;
    pv -= off;
    const bool row_in = pv >= 0 && pv < N;
    for (int qu = threadIdx.x; qu < npad; qu += blockDim.x) {
      int pu = qu + npad / 2;
      if (pu >= npad) pu -= npad;
      pu -= off;
      C out = cmake<C>(0.0, 0.0);
      if (row_in && pu >= 0 && pu < N) {
        const int64_t pix = static_cast<int64_t>(pv) * N + pu;
        double t = wb * omn[pix];
        t -= rint(t);
        T sn, cs;
        sincos_pi(static_cast<T>(2.0 * t), &sn, &cs);
        const T v = x[pix] * corr[pix];
        out.x = v * cs;
        out.y = v * sn;
      }
      grid[static_cast<int64_t>(qv) * npad + qu] = out;
    }
  }
}

// After the inverse FFTs of a group: x_p (+)= sum over its stacks of
// Re(conj(S~_k) G_k[P(p)]), one pass over the image per group.
template <typename T, typename C>
__global__ void finish_kernel(const C* __restrict__ grids, const double* __restrict__ omn,
                              const T* __restrict__ corr, int N, int npad,
                              const double* __restrict__ wbar, const int32_t* __restrict__ stacks,
                              int nslots, T* __restrict__ x, int accumulate) {
  const int off = (npad - N) / 2;
  const int64_t plane = static_cast<int64_t>(npad) * npad;
  for (int pv = blockIdx.x; pv < N; pv += gridDim.x) {
    int qv = pv + off + npad / 2;
    if (qv >= npad) qv -= npad;
    for (int pu = threadIdx.x; pu < N; pu += blockDim.x) {
      int qu = pu + off + npad / 2;
      if (qu >= npad) qu -= npad;
      const int64_t pix = static_cast<int64_t>(pv) * N + pu;
      const int64_t gi = static_cast<int64_t>(qv) * npad + qu;
      const double om = omn[pix];
      T acc = 0;
      for (int sl = 0; sl < nslots; ++sl) {
        const C g = grids[sl * plane + gi];
        double t = wbar[stacks[sl]] * om;
        t -= rint(t);
        T sn, cs;
        sincos_pi(static_cast<T>(2.0 * t), &sn, &cs);
        acc += cs * g.x + sn * g.y;
      }
      const T v = corr[pix] * acc;
      x[pix] = accumulate ? x[pix] + v : v;
    }
  }
}

// ---------------------------------------------------------------------------
// Deterministic gridding: fixed-point grid sums
// ---------------------------------------------------------------------------

// Per panel count P (thread P - 1): sum_j |w_K(j) 2 pi h g(r_j) r_j| over the
// P-panel node table.  With |chirp| = 1 and |J0| <= 1 every quadrature value
// of [GC] is bounded by it; the largest over P bounds them all.
template <typename T>
__global__ void kernel_bound_kernel(const T* __restrict__ hk, double* __restrict__ out) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (P > kMaxPanels) return;
  const int64_t off = panel_table_offset(P), n = static_cast<int64_t>(kNodes) * P;
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j) s += fabs(static_cast<double>(hk[off + j]));
  out[P - 1] = s;
}

// Largest term factor of one gridding call over records [0, n):
// |W_i| (|Re y_i| + |Im y_i|), times (sum_s |a_i(s)|)(sum_s |b_i(s)|) with a
// DDE, into *maxbits (the double's bits; non-negative doubles order as
// unsigned integers).  Any non-finite factor stores +Inf.
template <typename T, typename C>
__global__ void fixed_bound_kernel(const VisRec<T>* __restrict__ recs,
                                   const uint32_t* __restrict__ perm, int64_t n,
                                   const C* __restrict__ vis, const C* __restrict__ dde_a,
                                   const C* __restrict__ dde_b, int jd,
                                   unsigned long long* maxbits) {
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = perm[i] & 0x7fffffffu;
    const C y = vis[src];
    double f = fabs(static_cast<double>(recs[i].weight)) *
               (fabs(static_cast<double>(y.x)) + fabs(static_cast<double>(y.y)));
    if (dde_a) {
      double sa = 0.0, sb = 0.0;
      for (int j = 0; j < jd; ++j) {
        const C a = dde_a[src * jd + j], b = dde_b[src * jd + j];
        sa += fabs(static_cast<double>(a.x)) + fabs(static_cast<double>(a.y));
        sb += fabs(static_cast<double>(b.x)) + fabs(static_cast<double>(b.y));
      }
      f *= sa * sb;
    }
    m = isfinite(f) ? fmax(m, f) : HUGE_VAL;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(maxbits, static_cast<unsigned long long>(__double_as_longlong(m)));
}

// The exponent e of a call: every partial sum of a cell is at most
// n_terms * bound * max factor, and e keeps that below 2^61, within
// [emin, emax] (the range where 2^(32 - e) and 2^-e are numbers of the
// grid's precision); exp[1] = 1 for a non-finite factor.
__global__ void fixed_exp_kernel(const unsigned long long* __restrict__ maxbits, double scale,
                                 int emin, int emax, int* __restrict__ exp) {
  const double A = __longlong_as_double(static_cast<long long>(*maxbits)) * scale;
  if (!isfinite(A)) {
    exp[0] = 0;
    exp[1] = 1;
    return;
  }
  int ex = 0;
  if (A > 0.0) frexp(A, &ex);   // A < 2^ex
  exp[0] = min(max(61 - ex, emin), emax);
  exp[1] = 0;
}

// The fixed-point sums rounded into the complex grids (from_fixed), NaN
// throughout after a non-finite visibility.
template <typename T, typename C>
__global__ void fixed_to_grid_kernel(const longlong2* __restrict__ cells,
                                     const int* __restrict__ exp, int64_t n,
                                     C* __restrict__ grid) {
  const int e = exp[0];
  const bool bad = exp[1] != 0;
  const T s_hi = static_cast<T>(ldexp(1.0, 32 - e)), s_lo = static_cast<T>(ldexp(1.0, -e));
  const T nan = static_cast<T>(NAN);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const longlong2 v = cells[i];
    C out;
    out.x = bad ? nan : from_fixed(v.x, s_hi, s_lo);
    out.y = bad ? nan : from_fixed(v.y, s_hi, s_lo);
    grid[i] = out;
  }
}

// ---------------------------------------------------------------------------
// Fused kernel quadrature
// ---------------------------------------------------------------------------

// Build the weighted integrand values for panels [p0, p0 + np) of the
// npan-panel partition: h(r_j) e^{2 pi i dw (1 - n(r_j))}, phase argument in
// FP64, one NodeVal per node (FP64 path: Kronrod and difference weights).
template <typename T>
__device__ __forceinline__ void build_nodes(NodeVal<T>* sh, const QuadParams& q, int npan, int p0,
                                            int np, double dw, int lane) {
  const int64_t off = panel_table_offset(npan) + kNodes * (int64_t)p0;
  const double* omn = q.node_omn + off;
  const T* hk = static_cast<const T*>(q.node_hk) + off;
  const T* hd = static_cast<const T*>(q.node_hd) + off;
  for (int j = lane; j < kNodes * np; j += 32) {
    double t = dw * omn[j];
    t -= rint(t);
    T sn, cs;
    sincos_pi(static_cast<T>(2.0 * t), &sn, &cs);
    const T k = hk[j], d = hd[j];
    NodeVal<T> v;
    v.kr = k * cs;
    v.ki = k * sn;
    v.dr = d * cs;
    v.di = d * sn;
    sh[j] = v;
  }
}

// FP32 panels are evaluated two nodes at a time in Blackwell's paired FP32
// arithmetic, on the pairs of neighbouring nodes (2 k, 2 k + 1), k = 0..14,
// and node 30 alone.  A panel's values sit in kSlots float4 slots:
//   slot k (0..14)         {w_K h cos, w_K h sin} of the pair as
//                          {cos 2k, cos 2k+1, sin 2k, sin 2k+1};
//   slot 15 + k / 2        w_G h {cos, sin} of node 2 k + 1 (every odd node
//                          is a Gauss node) in components 2 (k & 1) + {0, 1};
//   slot 23                node 30: {w_K h cos, w_K h sin, 0, 0}.
// The FP32 node tables hold w_K h and w_G h (zero at Kronrod-only nodes).
constexpr int kPairs = (kNodes - 1) / 2;   // 15
constexpr int kSlots = 24;
static_assert(kSlots * 16 * kPanelBatch <= kNodeBatch * static_cast<int>(sizeof(NodeVal<float>)),
              "packed panels must fit the per-warp node buffer");

__device__ __forceinline__ void build_nodes(NodeVal<float>* sh, const QuadParams& q, int npan,
                                            int p0, int np, double dw, int lane) {
  const int64_t off = panel_table_offset(npan) + kNodes * (int64_t)p0;
  const double* omn = q.node_omn + off;
  const float* hk = static_cast<const float*>(q.node_hk) + off;
  const float* hg = static_cast<const float*>(q.node_hd) + off;
  float* shf = reinterpret_cast<float*>(sh);
  for (int j = lane; j < kNodes * np; j += 32) {
    double t = dw * omn[j];
    t -= rint(t);
    float sn, cs;
    sincospif(static_cast<float>(2.0 * t), &sn, &cs);
    const float k = hk[j], g = hg[j];
    const int p = j / kNodes, n = j - kNodes * p;
    float* base = shf + 4 * kSlots * p;
    if (n == kNodes - 1) {
      base[4 * 23] = k * cs;
      base[4 * 23 + 1] = k * sn;
      base[4 * 23 + 2] = 0.f;
      base[4 * 23 + 3] = 0.f;
    } else {
      const int pr = n >> 1, hi = n & 1;
      base[4 * pr + hi] = k * cs;
      base[4 * pr + 2 + hi] = k * sn;
      if (hi) {
        base[4 * (15 + (pr >> 1)) + 2 * (pr & 1)] = g * cs;
        base[4 * (15 + (pr >> 1)) + 2 * (pr & 1) + 1] = g * sn;
      }
    }
  }
}

// FP64 path: one rolled loop over the panel's nodes with CUDA's j0 for each
// of the lane's NT taps, the estimate summing |sum_j (w_K - w_G)_j f_j| per
// panel.
template <typename T, int NT>
__device__ __forceinline__ void eval_panels(const NodeVal<T>* sh, int p0, int np,
                                            const T (&Bh)[NT], T (&kr)[NT], T (&ki)[NT],
                                            T (&err)[NT]) {
  for (int p = 0; p < np; ++p) {
    const NodeVal<T>* hp = sh + kNodes * p;
    T a[NT], dr[NT], di[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      a[t] = Bh[t] * static_cast<T>(2 * (p0 + p) + 1);
      dr[t] = di[t] = 0;
    }
#pragma unroll 1
    for (int j = 0; j < kNodes; ++j) {
      const NodeVal<T> v = hp[j];
      const T x = gk_node_c(T(0), j);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const T J = j0_hc(fma(Bh[t], x, a[t]));
        kr[t] = fma(J, v.kr, kr[t]);
        ki[t] = fma(J, v.ki, ki[t]);
        dr[t] = fma(J, v.dr, dr[t]);
        di[t] = fma(J, v.di, di[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) err[t] += est_sqrt(dr[t] * dr[t] + di[t] * di[t]);
  }
}

// J0 regime of one node pair, the same for every lane of the warp: the
// degree-2 asymptotic form when the pair's lower node lies at u >= kJ0Far for
// every lane, the degree-4 form when it lies past J0's split, the
// small-argument series when the upper node lies below the split, and both
// (selected per node) otherwise.
enum PairRegime { kPairSmall = 0, kPairBoth = 1, kPairNear = 2, kPairFar = 3, kPairFarthest = 4 };

template <int kRegime>
__device__ __forceinline__ float2 j0_pair_regime(float2 u) {
  if (kRegime == kPairFarthest) return j0_farthest2(u);
  if (kRegime == kPairFar) return j0_far2(u);
  if (kRegime == kPairNear) return j0_large2(u);
  if (kRegime == kPairSmall) return j0_small2(u);
  const float2 Js = j0_small2(u), Jl = j0_large2(u);
  return make_float2(u.x > kJ0Split ? Jl.x : Js.x, u.y > kJ0Split ? Jl.y : Js.y);
}

// Pair k of one FP32 panel in regime R for each of the lane's NT taps: J0 at
// both nodes (x = node coordinates), the Kronrod sums, the Gauss sum of the
// odd node.  The node values v, g are loaded once for all NT taps.
template <int R, int NT>
__device__ __forceinline__ void panel_pair(float2 x, float4 v, float2 g, const float (&Bh)[NT],
                                           const float (&a)[NT], float2 (&KR)[NT],
                                           float2 (&KI)[NT], float (&gr)[NT], float (&gi)[NT]) {
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const float2 u = __ffma2_rn(x, make_float2(Bh[t], Bh[t]), make_float2(a[t], a[t]));
    const float2 J = j0_pair_regime<R>(u);
    KR[t] = __ffma2_rn(J, make_float2(v.x, v.y), KR[t]);
    KI[t] = __ffma2_rn(J, make_float2(v.z, v.w), KI[t]);
    gr[t] = fmaf(J.y, g.x, gr[t]);
    gi[t] = fmaf(J.y, g.y, gi[t]);
  }
}

// Pairs [k0, k1) of one FP32 panel in regime R, in a rolled loop (node
// coordinates from constant memory, values by computed index).
template <int R, int NT>
__device__ __forceinline__ void panel_pair_range(const float4* hp, int k0, int k1,
                                                 const float (&Bh)[NT], const float (&a)[NT],
                                                 float2 (&KR)[NT], float2 (&KI)[NT],
                                                 float (&gr)[NT], float (&gi)[NT]) {
  const float2* hg = reinterpret_cast<const float2*>(hp + 15);
#pragma unroll 1
  for (int k = k0; k < k1; ++k)
    panel_pair<R, NT>(make_float2(c_gk_node_f[2 * k], c_gk_node_f[2 * k + 1]), hp[k], hg[k], Bh,
                      a, KR, KI, gr, gi);
}

// One FP32 panel for the lane's NT taps.  kAllFar = kPairFarthest or
// kPairFar: every pair is in that regime (degree 1 or 2, unrolled);
// kAllFar = 0: pair k's regime follows from the warp-uniform counts ks (pairs
// all below the split), kn (pairs not all past it) and kf (pairs not all
// past kJ0Far), ks <= kn <= kf: the small-argument series below ks, both
// formulas below kn, degree 4 up to kf, degree 2 beyond, in short rolled
// loops.  Returns each tap's panel Kronrod sum (kr, ki) and Gauss sum (gr, gi).
template <int kAllFar, int NT>
__device__ __forceinline__ void panel_sums(const float4* hp, const float (&Bh)[NT],
                                           const float (&a)[NT], int ks, int kn, int kf,
                                           float (&kr)[NT], float (&ki)[NT], float (&gr)[NT],
                                           float (&gi)[NT]) {
  float2 KR[NT], KI[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    KR[t] = KI[t] = make_float2(0.f, 0.f);
    gr[t] = gi[t] = 0.f;
  }
  if (kAllFar) {
    // five pairs per loop trip: fully unrolled, the far panels' code alone
    // strained the instruction cache (1.5% slower per step)
    const float2* hg = reinterpret_cast<const float2*>(hp + 15);
#pragma unroll 5
    for (int k = 0; k < kPairs; ++k)
      panel_pair<kAllFar == kPairFarthest ? kPairFarthest : kPairFar, NT>(
          make_float2(c_gk_node_f[2 * k], c_gk_node_f[2 * k + 1]),
          hp[k], hg[k], Bh, a, KR, KI, gr, gi);
  } else {
    panel_pair_range<kPairSmall, NT>(hp, 0, ks, Bh, a, KR, KI, gr, gi);
    panel_pair_range<kPairBoth, NT>(hp, ks, kn, Bh, a, KR, KI, gr, gi);
    panel_pair_range<kPairNear, NT>(hp, kn, kf, Bh, a, KR, KI, gr, gi);
    panel_pair_range<kPairFar, NT>(hp, kf, kPairs, Bh, a, KR, KI, gr, gi);
  }
  // node 30, the panel's last
  const float4 c = hp[23];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const float u = fmaf(static_cast<float>(gk_node(kNodes - 1)), Bh[t], a[t]);
    const float J = kAllFar == kPairFarthest ? j0_farthest(u)
                    : (kAllFar || kf < kPairs) ? j0_far(u) : j0_halfcycles(u);
    kr[t] = fmaf(J, c.x, KR[t].x + KR[t].y);
    ki[t] = fmaf(J, c.y, KI[t].x + KI[t].y);
  }
}

// FP32: per panel, the Kronrod sum K_p and the Gauss sum G_p of each of the
// lane's NT taps; the estimate adds |K_p - G_p|, formed from the panel's own
// sums (of the panel's size, not the whole integral's).  The J0 regime of
// each node pair follows from the smallest and largest Bh of the warp's
// active taps (warp-uniform): node j of panel P lies at u = Bh (2 P + 1 + x_j)
// for each tap.
template <int NT>
__device__ __forceinline__ void eval_panels_f32(const NodeVal<float>* sh, int p0, int np,
                                                const float (&Bh)[NT], float bh_min,
                                                float bh_max, float (&kr)[NT], float (&ki)[NT],
                                                float (&err)[NT]) {
  const float4* hp = reinterpret_cast<const float4*>(sh);
  const int lane = threadIdx.x & 31;
  float f = static_cast<float>(2 * p0 + 1);   // 2 (p0 + p) + 1, exact
  for (int p = 0; p < np; ++p, f += 2.f, hp += kSlots) {
    float a[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) a[t] = Bh[t] * f;
    float pkr[NT], pki[NT], pgr[NT], pgi[NT];
    const float lo_min = bh_min * (f + c_gk_node_f[0]);   // lowest node of any tap
    if (lo_min >= kJ0Farthest) {
      panel_sums<kPairFarthest, NT>(hp, Bh, a, 0, 0, 0, pkr, pki, pgr, pgi);
    } else if (lo_min >= kJ0Far) {
      panel_sums<kPairFar, NT>(hp, Bh, a, 0, 0, 0, pkr, pki, pgr, pgi);
    } else {
      // lane k < 15 classifies pair k; the counts are the same in every lane
      const bool on = lane < kPairs;
      const float tlo = f + c_gk_node_f[on ? 2 * lane : 0];
      const float thi = f + c_gk_node_f[on ? 2 * lane + 1 : 0];
      const int kf = __popc(__ballot_sync(0xffffffffu, on && !(bh_min * tlo >= kJ0Far)));
      const int kn = __popc(__ballot_sync(0xffffffffu, on && !(bh_min * tlo > kJ0Split)));
      const int ks = __popc(__ballot_sync(0xffffffffu, on && bh_max * thi <= kJ0Split));
      panel_sums<0, NT>(hp, Bh, a, ks, kn, kf, pkr, pki, pgr, pgi);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      kr[t] += pkr[t];
      ki[t] += pki[t];
      const float dr = pkr[t] - pgr[t], di = pki[t] - pgi[t];
      err[t] += est_sqrt(dr * dr + di * di);
    }
  }
}

// The FP32 quadrature of eval_chunk for NT taps per lane (a chunk of 32 NT
// taps): one node build, one panel schedule and one refinement decision for
// all of them.
template <int NT, typename N>
__device__ __forceinline__ void eval_chunk_f32(NodeVal<float>* sh, const QuadParams& q,
                                               const float (&rho)[NT], const bool (&active)[NT],
                                               double dw, int npan, int max_panels, int& built,
                                               bool (&ok)[NT], int lane, N& nodes,
                                               float2 (&K)[NT]) {
  npan = min(npan, max_panels);
  // the active taps' extreme radii (warp-uniform)
  float rmin = 1e30f, rmax = 0.f;
#pragma unroll
  for (int t = 0; t < NT; ++t)
    if (active[t]) {
      rmin = fminf(rmin, rho[t]);
      rmax = fmaxf(rmax, rho[t]);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  int refine = 0;
  while (true) {
    const float hb = q.Rf / static_cast<float>(npan);
    float Bh[NT], kr[NT], ki[NT], err[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      nodes += active[t] ? static_cast<N>(kNodes * npan) : N(0);
      Bh[t] = hb * rho[t];
      kr[t] = ki[t] = err[t] = 0.f;
    }
    if (npan <= kPanelBatch) {
      if (built != npan) {
        __syncwarp();
        build_nodes(sh, q, npan, 0, npan, dw, lane);
        __syncwarp();
        built = npan;
      }
      eval_panels_f32<NT>(sh, 0, npan, Bh, hb * rmin, hb * rmax, kr, ki, err);
    } else {
      for (int p0 = 0; p0 < npan; p0 += kPanelBatch) {
        const int nb = min(kPanelBatch, npan - p0);
        __syncwarp();
        build_nodes(sh, q, npan, p0, nb, dw, lane);
        __syncwarp();
        eval_panels_f32<NT>(sh, p0, nb, Bh, hb * rmin, hb * rmax, kr, ki, err);
      }
      built = 0;
    }
    bool bad = false;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float lim = fmaxf(q.tol_abs, q.tol_rel * est_sqrt(kr[t] * kr[t] + ki[t] * ki[t]));
      ok[t] = (!active[t]) || err[t] <= lim;
      bad = bad || !ok[t];
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (!any_bad || refine >= q.max_refine || npan >= max_panels) {
#pragma unroll
      for (int t = 0; t < NT; ++t) K[t] = make_float2(kr[t], ki[t]);
      return;
    }
    ++refine;
    npan = min(2 * npan, max_panels);
  }
}

// Half-cycles of J0 per unit node coordinate for a tap at rho on npan
// panels: 2 rho R / (2 npan) (the FP32 path forms (R / npan) rho in FP32).
__device__ __forceinline__ double panel_bh(const QuadParams& q, double rho, int npan) {
  return (q.R / npan) * rho;
}

// eval_chunk's FP64 path for NT taps per lane: one NodeVal per node.
template <int NT, typename T, typename C, typename N>
__device__ __forceinline__ void eval_chunk_generic(NodeVal<T>* sh, const QuadParams& q,
                                                   const T (&rho)[NT], const bool (&active)[NT],
                                                   double dw, int npan, int max_panels,
                                                   int& built, bool (&ok)[NT], int lane,
                                                   N& nodes, C (&K)[NT]) {
  npan = min(npan, max_panels);
  int refine = 0;
  while (true) {
    T Bh[NT], kr[NT], ki[NT], err[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      nodes += active[t] ? static_cast<N>(kNodes * npan) : N(0);
      Bh[t] = panel_bh(q, rho[t], npan);
      kr[t] = ki[t] = err[t] = 0;
    }
    if (npan <= kPanelBatch) {
      if (built != npan) {
        __syncwarp();
        build_nodes(sh, q, npan, 0, npan, dw, lane);
        __syncwarp();
        built = npan;
      }
      eval_panels<T, NT>(sh, 0, npan, Bh, kr, ki, err);
    } else {
      for (int p0 = 0; p0 < npan; p0 += kPanelBatch) {
        const int nb = min(kPanelBatch, npan - p0);
        __syncwarp();
        build_nodes(sh, q, npan, p0, nb, dw, lane);
        __syncwarp();
        eval_panels<T, NT>(sh, p0, nb, Bh, kr, ki, err);
      }
      built = 0;
    }
    bool bad = false;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const T lim = fmax(static_cast<T>(q.tol_abs),
                         static_cast<T>(q.tol_rel) * est_sqrt(kr[t] * kr[t] + ki[t] * ki[t]));
      ok[t] = (!active[t]) || err[t] <= lim;
      bad = bad || !ok[t];
    }
    const bool any_bad = __any_sync(0xffffffffu, bad);
    if (!any_bad || refine >= q.max_refine || npan >= max_panels) {
#pragma unroll
      for (int t = 0; t < NT; ++t) K[t] = cmake<C>(kr[t], ki[t]);
      return;
    }
    ++refine;
    npan = min(2 * npan, max_panels);
  }
}

// [GC] for NT taps per lane of a chunk of 32 NT taps, in the precision T.
template <int NT, typename T, typename C, typename N>
__device__ __forceinline__ void eval_chunk_nt(NodeVal<T>* sh, const QuadParams& q,
                                              const T (&rho)[NT], const bool (&active)[NT],
                                              double dw, int npan, int max_panels, int& built,
                                              bool (&ok)[NT], int lane, N& nodes, C (&K)[NT]) {
  if constexpr (sizeof(T) == 4)
    eval_chunk_f32<NT>(sh, q, rho, active, dw, npan, max_panels, built, ok, lane, nodes, K);
  else
    eval_chunk_generic<NT>(sh, q, rho, active, dw, npan, max_panels, built, ok, lane, nodes, K);
}

// Evaluate [GC](rho, dw) for one tap per lane (inactive lanes compute a
// harmless dummy) on npan panels, doubling the panels for the whole chunk
// while any active tap misses the tolerance, up to max_panels (the node
// tables' largest partition) and max_refine doublings.  `built` (the panel
// count whose nodes are resident in sh, or 0) is warp-uniform and updated.
template <typename T, typename C, typename N>
__device__ __forceinline__ C eval_chunk(NodeVal<T>* sh, const QuadParams& q, T rho, bool active,
                                        double dw, int npan, int max_panels, int& built, bool& ok,
                                        int lane, N& nodes) {
  const T r1[1] = {rho};
  const bool a1[1] = {active};
  bool ok1[1];
  C K1[1];
  eval_chunk_nt<1>(sh, q, r1, a1, dw, npan, max_panels, built, ok1, lane, nodes, K1);
  ok = ok1[0];
  return K1[0];
}

// ---------------------------------------------------------------------------
// Pieces shared by the per-visibility kernels
// ---------------------------------------------------------------------------

// A warp's share of the work queue: visibilities are claimed `batch` at a
// time from the shared head (one atomic per batch).  take() is false once the
// queue is empty.
struct WarpQueue {
  unsigned long long next = 0, stop = 0;
  __device__ __forceinline__ bool take(unsigned long long* head, unsigned long long batch,
                                       int64_t n, int lane, unsigned long long& i) {
    if (next == stop) {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(head, batch);
      i0 = __shfl_sync(0xffffffffu, i0, 0);
      next = i0;
      stop = min(i0 + batch, static_cast<unsigned long long>(n));
      if (next >= stop) return false;
    }
    i = next++;
    return true;
  }
};

// The value a gridded visibility spreads: W_i y_i, conjugated back if folded.
template <typename T, typename C>
__device__ __forceinline__ C load_visibility(const C* __restrict__ vis_in, uint32_t pm, T weight) {
  C v = vis_in[pm & 0x7fffffffu];
  if (pm >> 31) v.y = -v.y;
  v.x *= weight;
  v.y *= weight;
  return v;
}

// One tap: gridding adds conj(K) yv to the grid cell, degridding accumulates
// K times the cell.
template <typename C, bool kGrid>
__device__ __forceinline__ void apply_tap(const C& K, int64_t gi, const C& yv,
                                          const C* __restrict__ grid_in, C* grid_out,
                                          const FixedGrid& fx, C& accv) {
  if (kGrid) {
    C add;
    add.x = K.x * yv.x + K.y * yv.y;   // conj(K) * yv
    add.y = K.x * yv.y - K.y * yv.x;
    grid_add(grid_out, fx, gi, add);
  } else {
    const C g = grid_in[gi];
    accv.x += K.x * g.x - K.y * g.y;
    accv.y += K.x * g.y + K.y * g.x;
  }
}

// Degridding: the warp's tap sums reduced, weighted, conjugated if folded and
// stored in the caller's order.
template <typename T, typename C>
__device__ __forceinline__ void store_visibility(C accv, T weight, uint32_t pm,
                                                 C* __restrict__ vis_out, int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    accv.x += __shfl_xor_sync(0xffffffffu, accv.x, o);
    accv.y += __shfl_xor_sync(0xffffffffu, accv.y, o);
  }
  if (lane == 0) {
    C out;
    out.x = accv.x * weight;
    out.y = accv.y * weight;
    if (pm >> 31) out.y = -out.y;
    vis_out[pm & 0x7fffffffu] = out;
  }
}

// The warp's counters into the plan's statistics: [0] unconverged, [1] taps,
// [3] tap-node evaluations.
__device__ __forceinline__ void flush_counts(unsigned long long* stats, unsigned long long bad,
                                             unsigned long long taps, unsigned long long nodes,
                                             int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
    taps += __shfl_xor_sync(0xffffffffu, taps, o);
    nodes += __shfl_xor_sync(0xffffffffu, nodes, o);
  }
  if (lane == 0 && taps) {
    if (bad) atomicAdd(stats, bad);
    atomicAdd(stats + 1, taps);
    if (nodes) atomicAdd(stats + 3, nodes);
  }
}

// Panels for the chunk: integrand cycles over [0, R] bounded by
// R (rho_max + |dw| chirp_coeff), at inv_cycles panels per cycle.
__device__ __forceinline__ int initial_panels(const QuadParams& q, float rho_max, float adw) {
  return panel_count_for(q.Rf * fmaf(adw, q.chirp_coeff, rho_max) * q.inv_cycles);
}

// Taps per lane of the fused kernel's chunks.
constexpr int kVisTaps = 2;

// Block shape of the fused kernel: threads per block and the blocks per SM
// its register budget is sized for (FP32: 4 x 256 threads, 64 registers;
// 7 x 128 threads at 72 registers and 3 x 256 at 80 ran slower).
template <typename T> struct VisLaunch {
  static constexpr int threads = 256;
  static constexpr int min_blocks = sizeof(T) == 4 ? 4 : 2;
};

// One warp per visibility, visibilities taken from a work queue.  Taps are
// visited in order of distance from the box centre, 32 kVisTaps at a time;
// each chunk takes the panel count its farthest tap needs.
template <typename T, typename C, bool kGrid>
__global__ void __launch_bounds__(VisLaunch<T>::threads, VisLaunch<T>::min_blocks)
    vis_kernel(const VisRec<T>* __restrict__ recs, const uint32_t* __restrict__ perm, int64_t n,
               const C* __restrict__ grid_in, C* grid_out, const C* __restrict__ vis_in,
               C* __restrict__ vis_out, QuadParams q, const int32_t* __restrict__ stack_slot,
               unsigned long long* head, unsigned long long* stats, int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  unsigned long long my_bad = 0, my_taps = 0, my_nodes = 0;
  const int npad = q.npad;
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    const int Jw = r.jw;
    // the grid of this visibility's stack within the resident group
    const int64_t gbase = static_cast<int64_t>(stack_slot[r.stack]) * npad * npad;
    const int half = Jw / 2;
    const T fu = r.fu, fv = r.fv;
    const uint16_t* order = q.tap_order + q.tap_off[half - 1];
    const float adw = static_cast<float>(fabs(r.dw));
    int built = 0;
    const uint32_t pm = perm[i];
    const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                       : cmake<C>(0.0, 0.0);
    C accv = cmake<C>(0.0, 0.0);
    const int ntap = Jw * Jw;
    // kVisTaps taps per lane: a chunk of 32 kVisTaps consecutive taps shares
    // one node build, panel schedule and refinement decision
    for (int t0 = 0; t0 < ntap; t0 += 32 * kVisTaps) {
      T rho[kVisTaps];
      bool act[kVisTaps], ok[kVisTaps];
      uint32_t code[kVisTaps];
      T rmax = T(0);
#pragma unroll
      for (int k = 0; k < kVisTaps; ++k) {
        const int t = t0 + 32 * k + lane;
        act[k] = t < ntap;
        code[k] = order[act[k] ? t : 0];
        const T du_ = fu - static_cast<T>(static_cast<int>(code[k] & 0xffu) - half + 1);
        const T dv_ = fv - static_cast<T>(static_cast<int>(code[k] >> 8) - half + 1);
        rho[k] = sqrt(du_ * du_ + dv_ * dv_);
        if (act[k]) rmax = fmax(rmax, rho[k]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      const int npan = initial_panels(q, static_cast<float>(rmax), adw);
      C K[kVisTaps];
      eval_chunk_nt<kVisTaps>(sh, q, rho, act, r.dw, npan, kMaxPanels, built, ok, lane, my_nodes,
                              K);
#pragma unroll
      for (int k = 0; k < kVisTaps; ++k)
        if (act[k]) {
          if (!ok[k]) ++my_bad;
          const int ou = static_cast<int>(code[k] & 0xffu) - half + 1;
          const int ov = static_cast<int>(code[k] >> 8) - half + 1;
          const int64_t gi = gbase + static_cast<int64_t>(wrap_index(r.bv + ov, npad)) * npad +
                             wrap_index(r.bu + ou, npad);
          apply_tap<C, kGrid>(K[k], gi, yv, grid_in, grid_out, q.fx, accv);
        }
    }
    if (lane == 0) my_taps += static_cast<unsigned long long>(ntap);
    if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
  }
  flush_counts(stats, my_bad, my_taps, my_nodes, lane);
}

// ---------------------------------------------------------------------------
// Pre-sampled 1-D w-planes (Sec. 5.1.1)
// ---------------------------------------------------------------------------

// Two adjacent w-planes at one radius: {K(j, i), K(j + 1, i)}.
template <typename C> struct __align__(2 * sizeof(C)) KPair { C a, b; };

// Sample K(i h_rho, j h_w) for all i < nr, j < nw: one warp per w-plane,
// lanes over radii, 32 radii per chunk sharing one node set (the same
// quadrature routine as the degridder).
template <typename T, typename C>
__global__ void __launch_bounds__(256) table_sample_kernel(C* __restrict__ raw, int64_t nr,
                                                           int64_t nw, double hr, double hw,
                                                           QuadParams q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  const int64_t wpb = blockDim.x >> 5;
  unsigned long long nodes = 0;
  for (int64_t j = blockIdx.x * wpb + warp; j < nw; j += (int64_t)gridDim.x * wpb) {
    const double w = static_cast<double>(j) * hw;
    int built = 0;
    for (int64_t i0 = 0; i0 < nr; i0 += 32) {
      const int64_t i = i0 + lane;
      const bool active = i < nr;
      const T rho = static_cast<T>(static_cast<double>(active ? i : i0) * hr);
      const int64_t ilast = min(i0 + 31, nr - 1);
      const int npan = initial_panels(q, static_cast<float>(ilast * hr), static_cast<float>(w));
      bool ok = true;
      const C K = eval_chunk<T, C>(sh, q, rho, active, w, npan, kMaxPanels, built, ok, lane, nodes);
      if (active) raw[j * nr + i] = K;
    }
  }
}

// Pair entries for w-row j at radius i: {K(j, i), K(j + 1, i) - K(j, i)}.
template <typename C>
__global__ void table_pair_kernel(const C* __restrict__ raw, int64_t nr, int64_t nw,
                                  KPair<C>* __restrict__ pairs) {
  const int64_t total = (nw - 1) * nr;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const C lo = raw[k], hi = raw[k + nr];
    KPair<C> v;
    v.a = lo;
    v.b.x = hi.x - lo.x;
    v.b.y = hi.y - lo.y;
    pairs[k] = v;
  }
}

// The tabulated kernel between radius samples i (p0) and i + 1 (p1) at
// fractions fr (radius) and fw (w-row): linear in |dw| at each radius, then
// linear in rho.
template <typename T, typename C>
__device__ __forceinline__ C table_interp(const KPair<C>& p0, const KPair<C>& p1, T fr, T fw) {
  const T k0x = fma(fw, p0.b.x, p0.a.x), k0y = fma(fw, p0.b.y, p0.a.y);
  const T k1x = fma(fw, p1.b.x, p1.a.x), k1y = fma(fw, p1.b.y, p1.a.y);
  C K;
  K.x = fma(fr, k1x - k0x, k0x);
  K.y = fma(fr, k1y - k0y, k0y);
  return K;
}

// Table position of a tap at (du, dv) cells from the visibility: s =
// |(du, dv)| / h_rho.  FP32 takes the hardware square root (relative error
// about 2^-22, far below the table's interpolation error); FP64 the
// correctly rounded one.
__device__ __forceinline__ float table_radius(float du, float dv, float inv_hr) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fmaf(du, du, dv * dv)));
  return r * inv_hr;
}
__device__ __forceinline__ double table_radius(double du, double dv, double inv_hr) {
  return sqrt(fma(du, du, dv * dv)) * inv_hr;
}

// The taps of one visibility from the plane pair of its w-row (`row`, in
// shared or global memory), raster order, 32 at a time; tap t = b J_w + a is
// advanced by 32 per step without a division, the offsets also kept as
// floats so that no tap needs an int <-> float conversion (those run on the
// FP64 unit here).  kContig: the box lies inside the grid without wrapping
// (warp-uniform) and `grid` points at its first cell, so tap (a, b) is cell
// b npad + a; otherwise `grid` is the stack's grid and each tap wraps its own
// indices.  The conjugation for dw < 0 is left to the caller: with K = Kx +
// i s Ky, degridding sums Kx g (sx) and Ky g (sy) apart, gridding adds
// Kx yv + Ky ys with ys = -i s yv.
template <bool kContig, bool kGrid, typename T, typename C>
__device__ __forceinline__ void table_vis_taps(const KPair<C>* __restrict__ row,
                                               const VisRec<T>& r, T fw, int nr, T inv_hr,
                                               int npad, const C* __restrict__ grid_in,
                                               C* grid_out, const FixedGrid& fx, C yv, C ys,
                                               C& sx, C& sy, int lane) {
  const int Jw = r.jw, half = Jw / 2, ntap = Jw * Jw;
  const T last_r = static_cast<T>(nr - 2);
  int a = lane % Jw, b = lane / Jw;
  const int step_b = 32 / Jw, step_a = 32 % Jw;
  T du_ = r.fu - static_cast<T>(a - half + 1), dv_ = r.fv - static_cast<T>(b - half + 1);
  const T fstep_a = static_cast<T>(step_a), fstep_b = static_cast<T>(step_b);
  const T fJw = static_cast<T>(Jw);
  int off = b * npad + a;
  const int step_off = step_b * npad + step_a, carry_off = npad - Jw;
#pragma unroll 4
  for (int t0 = 0; t0 < ntap; t0 += 32) {
    int ir;
    T fr;
    table_index(table_radius(du_, dv_, inv_hr), nr - 2, last_r, ir, fr);
    const C K = table_interp<T, C>(row[ir], row[ir + 1], fr, fw);
    int64_t gi;
    if (kContig) {
      gi = off;
    } else {
      gi = static_cast<int64_t>(wrap_index(r.bv + b - half + 1, npad)) * npad +
           wrap_index(r.bu + a - half + 1, npad);
    }
    if (t0 + lane < ntap) {
      if (kGrid) {
        C add;
        add.x = fma(K.x, yv.x, K.y * ys.x);
        add.y = fma(K.x, yv.y, K.y * ys.y);
        grid_add(grid_out, fx, gi, add);
      } else {
        const C g = grid_in[gi];
        sx.x = fma(K.x, g.x, sx.x);
        sx.y = fma(K.x, g.y, sx.y);
        sy.x = fma(K.y, g.x, sy.x);
        sy.y = fma(K.y, g.y, sy.y);
      }
    }
    a += step_a;
    b += step_b;
    du_ -= fstep_a;
    dv_ -= fstep_b;
    off += step_off;
    if (a >= Jw) {
      a -= Jw;
      ++b;
      du_ += fJw;
      dv_ -= T(1);
      off += carry_off;
    }
  }
}

// One visibility of a table kernel: the box's placement on the grid, the
// conjugation for dw < 0 and the tap loop; degridding returns the lane's
// partial sum.
template <bool kGrid, typename T, typename C>
__device__ __forceinline__ C table_vis(const KPair<C>* __restrict__ row, const VisRec<T>& r,
                                       T fw, int nr, T inv_hr, int npad,
                                       const C* __restrict__ grid_in, C* grid_out,
                                       const FixedGrid& fx, C yv, int lane) {
  const int Jw = r.jw, half = Jw / 2;
  const T sg = r.dw < 0.0 ? T(-1) : T(1);
  C ys;
  ys.x = sg * yv.y;
  ys.y = -sg * yv.x;
  C sx = cmake<C>(0.0, 0.0), sy = cmake<C>(0.0, 0.0);
  const int u0 = wrap_index(r.bu - half + 1, npad), v0 = wrap_index(r.bv - half + 1, npad);
  if (u0 + Jw <= npad && v0 + Jw <= npad) {
    const int64_t o0 = static_cast<int64_t>(v0) * npad + u0;
    table_vis_taps<true, kGrid>(row, r, fw, nr, inv_hr, npad, kGrid ? nullptr : grid_in + o0,
                                kGrid ? grid_out + o0 : nullptr, fixed_offset(fx, o0), yv, ys,
                                sx, sy, lane);
  } else {
    table_vis_taps<false, kGrid>(row, r, fw, nr, inv_hr, npad, grid_in, grid_out, fx, yv, ys,
                                 sx, sy, lane);
  }
  C acc;   // sum of (Kx + i s Ky) g
  acc.x = fma(-sg, sy.y, sx.x);
  acc.y = fma(sg, sy.x, sx.y);
  return acc;
}

// Degrid / grid with every tap interpolated bilinearly in (rho, |dw|) from
// the pre-sampled w-planes, conjugated for dw < 0.  One warp per visibility
// (its two w-planes stay in L1 while its taps are read), taps in raster order.
template <typename T, typename C, bool kGrid>
__global__ void __launch_bounds__(256) vis_table_kernel(const VisRec<T>* __restrict__ recs,
                                                        const uint32_t* __restrict__ perm,
                                                        int64_t n, const C* __restrict__ grid_in,
                                                        C* grid_out, const C* __restrict__ vis_in,
                                                        C* __restrict__ vis_out, TableView<T> tv,
                                                        int npad_i,
                                                        const int32_t* __restrict__ stack_slot,
                                                        unsigned long long* head,
                                                        unsigned long long* stats, int batch) {
  const int lane = threadIdx.x & 31;
  const KPair<C>* __restrict__ pairs = static_cast<const KPair<C>*>(tv.pairs);
  const int npad = npad_i;
  const int nr = static_cast<int>(tv.nr), nw = static_cast<int>(tv.nw);
  unsigned long long my_taps = 0;
  // batches of visibilities: with small supports a visibility is cheap and
  // one atomic per visibility on the shared queue head would serialise warps
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    // the grid of this visibility's stack within the resident group
    const int64_t gbase = static_cast<int64_t>(stack_slot[r.stack]) * npad * npad;
    const T aw = table_w_scaled(static_cast<T>(fabs(r.dw)), tv.inv_hw);
    const int jrow = table_w_row(aw, nw - 2);
    const T fw = aw - static_cast<T>(jrow);
    const uint32_t pm = perm[i];
    const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                       : cmake<C>(0.0, 0.0);
    const C accv = table_vis<kGrid>(pairs + static_cast<int64_t>(jrow) * nr, r, fw, nr,
                                    tv.inv_hr, npad, kGrid ? nullptr : grid_in + gbase,
                                    kGrid ? grid_out + gbase : nullptr,
                                    fixed_offset(tv.fx, gbase), yv, lane);
    if (lane == 0) my_taps += static_cast<unsigned long long>(r.jw * r.jw);
    if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
  }
  flush_counts(stats, 0, my_taps, 0, lane);
}

// Degrid / grid with the tabulated kernel, one thread block per uv-tile work
// item.  The block stages the item's grid patch -- the tile plus J_w - 1
// cells of halo, wrapped circularly -- in shared memory: degridding reads
// every tap from the patch; gridding accumulates into the zeroed patch with
// shared-memory atomics and adds the patch to the grid once, with one global
// atomic per non-zero cell instead of one per tap.
template <typename T, typename C, bool kGrid>
__global__ void __launch_bounds__(256) tile_table_kernel(
    const VisRec<T>* __restrict__ recs, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ item_se, const uint32_t* __restrict__ item_key, int n_items,
    const C* __restrict__ grids_in, C* grids_out, const C* __restrict__ vis_in,
    C* __restrict__ vis_out, TableView<T> tv, int npad, int tile, int tiles_per_row, int jmax,
    const int32_t* __restrict__ stack_slot, unsigned long long* head, unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* patch = reinterpret_cast<C*>(smem_raw);
  __shared__ int s_item;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int side = tile + jmax;
  const KPair<C>* __restrict__ pairs = static_cast<const KPair<C>*>(tv.pairs);
  const int nr = static_cast<int>(tv.nr), nw = static_cast<int>(tv.nw);
  const T last_r = static_cast<T>(nr - 2);
  unsigned long long my_taps = 0;
  while (true) {
    if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(head, 1ULL));
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int64_t gbase =
        static_cast<int64_t>(stack_slot[item_key[item] >> 24]) * npad * npad;
    const C* __restrict__ grid_in = kGrid ? nullptr : grids_in + gbase;
    C* grid_out = kGrid ? grids_out + gbase : nullptr;
    const uint32_t key = item_key[item] & 0xffffffu;
    const int tu = static_cast<int>(key % tiles_per_row), tvv = static_cast<int>(key / tiles_per_row);
    const int u0 = tu * tile - npad / 2 - jmax / 2 + 1;
    const int v0 = tvv * tile - npad / 2 - jmax / 2 + 1;
    for (int c = threadIdx.x; c < side * side; c += blockDim.x) {
      const int pv = c / side, pu = c - pv * side;
      if (kGrid) {
        patch[c] = cmake<C>(0.0, 0.0);
      } else {
        patch[c] = grid_in[static_cast<int64_t>(wrap_index(v0 + pv, npad)) * npad +
                           wrap_index(u0 + pu, npad)];
      }
    }
    __syncthreads();
    const int r0 = item_se[2 * item], r1 = item_se[2 * item + 1];
    for (int ri = r0 + warp; ri < r1; ri += nwarps) {
      const VisRec<T> r = recs[ri];
      const int Jw = r.jw;
      const int half = Jw / 2;
      const T aw = table_w_scaled(static_cast<T>(fabs(r.dw)), tv.inv_hw);
      const int jrow = table_w_row(aw, nw - 2);
      const T fw = aw - static_cast<T>(jrow);
      const bool neg = r.dw < 0.0;
      const KPair<C>* row = pairs + static_cast<int64_t>(jrow) * nr;
      const uint32_t pm = perm[ri];
      const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                         : cmake<C>(0.0, 0.0);
      // patch position of tap (0, 0) = (bu - half + 1, bv - half + 1)
      const int pu0 = r.bu - half + 1 - u0, pv0 = r.bv - half + 1 - v0;
      C accv = cmake<C>(0.0, 0.0);
      const int ntap = Jw * Jw;
      int a = lane % Jw, b = lane / Jw;
      const int step_b = 32 / Jw, step_a = 32 % Jw;
      T du_ = r.fu - static_cast<T>(a - half + 1), dv_ = r.fv - static_cast<T>(b - half + 1);
      const T fstep_a = static_cast<T>(step_a), fstep_b = static_cast<T>(step_b);
      const T fJw = static_cast<T>(Jw);
      for (int t0 = 0; t0 < ntap; t0 += 32) {
        if (t0 + lane < ntap) {
          int ir;
          T fr;
          table_index(table_radius(du_, dv_, tv.inv_hr), nr - 2, last_r, ir, fr);
          C K = table_interp<T, C>(row[ir], row[ir + 1], fr, fw);
          if (neg) K.y = -K.y;
          const int li = (pv0 + b) * side + (pu0 + a);
          if (kGrid) {
            atomicAdd(&patch[li].x, K.x * yv.x + K.y * yv.y);   // conj(K) * yv
            atomicAdd(&patch[li].y, K.x * yv.y - K.y * yv.x);
          } else {
            const C g = patch[li];
            accv.x += K.x * g.x - K.y * g.y;
            accv.y += K.x * g.y + K.y * g.x;
          }
        }
        a += step_a;
        b += step_b;
        du_ -= fstep_a;
        dv_ -= fstep_b;
        if (a >= Jw) {
          a -= Jw;
          ++b;
          du_ += fJw;
          dv_ -= T(1);
        }
      }
      if (lane == 0) my_taps += static_cast<unsigned long long>(ntap);
      if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
    }
    __syncthreads();
    if (kGrid) {
      for (int c = threadIdx.x; c < side * side; c += blockDim.x) {
        const C v = patch[c];
        if (v.x != T(0) || v.y != T(0)) {
          const int pv = c / side, pu = c - pv * side;
          atomic_add_c(grid_out + static_cast<int64_t>(wrap_index(v0 + pv, npad)) * npad +
                           wrap_index(u0 + pu, npad),
                       v);
        }
      }
      __syncthreads();
    }
  }
  flush_counts(stats, 0, my_taps, 0, lane);
}

// Degrid / grid with the tabulated kernel, one thread block per w-row work
// item (grid_staging 2): the block copies the item's pair of adjacent
// w-planes, all n_rho radii, into shared memory once, then its warps take the
// item's visibilities (every kept visibility whose |dw| falls on that row)
// one at a time and read both entries of every tap from shared memory.  A
// tap's 16-byte table entries are scattered over the row, one cache line
// each from global memory; from shared memory they cost a bank access.  The
// taps, their order and arithmetic are those of vis_table_kernel.
template <typename T, typename C, bool kGrid>
__global__ void __launch_bounds__(256) row_table_kernel(
    const VisRec<T>* __restrict__ recs, const uint32_t* __restrict__ perm,
    const uint32_t* __restrict__ row_idx, const int32_t* __restrict__ item_se,
    const uint32_t* __restrict__ item_key, int n_items, const C* __restrict__ grid_in,
    C* grid_out, const C* __restrict__ vis_in, C* __restrict__ vis_out, TableView<T> tv,
    int npad, const int32_t* __restrict__ stack_slot, unsigned long long* head,
    unsigned long long* stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  KPair<C>* row = reinterpret_cast<KPair<C>*>(smem_raw);
  __shared__ int s_item;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const KPair<C>* __restrict__ pairs = static_cast<const KPair<C>*>(tv.pairs);
  const int nr = static_cast<int>(tv.nr);
  unsigned long long my_taps = 0;
  while (true) {
    if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(head, 1ULL));
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int jrow = static_cast<int>(item_key[item] & 0xffffffu);
    const KPair<C>* src = pairs + static_cast<int64_t>(jrow) * nr;
    for (int c = threadIdx.x; c < nr; c += blockDim.x) row[c] = src[c];
    __syncthreads();
    const int r0 = item_se[2 * item], r1 = item_se[2 * item + 1];
    for (int ri = r0 + warp; ri < r1; ri += nwarps) {
      const uint32_t rec = row_idx[ri];
      const VisRec<T> r = recs[rec];
      const int64_t gbase = static_cast<int64_t>(stack_slot[r.stack]) * npad * npad;
      // the item's row is this record's (the plan keyed it with the same
      // arithmetic), so fw lies in [0, 1]
      const T fw = table_w_scaled(static_cast<T>(fabs(r.dw)), tv.inv_hw) - static_cast<T>(jrow);
      const uint32_t pm = perm[rec];
      const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                         : cmake<C>(0.0, 0.0);
      const C accv = table_vis<kGrid>(row, r, fw, nr, tv.inv_hr, npad,
                                      kGrid ? nullptr : grid_in + gbase,
                                      kGrid ? grid_out + gbase : nullptr,
                                      fixed_offset(tv.fx, gbase), yv, lane);
      if (lane == 0) my_taps += static_cast<unsigned long long>(r.jw * r.jw);
      if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
    }
    __syncthreads();   // the row is rewritten by the next item
  }
  flush_counts(stats, 0, my_taps, 0, lane);
}

// phi_wkernel: one warp per point, lane 0 carries the tap.
template <typename T, typename C>
__global__ void __launch_bounds__(256) wkernel_kernel(const double* __restrict__ rho_in,
                                                      const double* __restrict__ dw_in, int64_t n,
                                                      C* __restrict__ out, QuadParams q,
                                                      unsigned long long* bad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = blockIdx.x * wpb + warp; i < n; i += (int64_t)gridDim.x * wpb) {
    const T rho = static_cast<T>(rho_in[i]);
    const double dw = dw_in[i];
    int built = 0;
    bool ok = true;
    unsigned long long nodes = 0;
    const C K = eval_chunk<T, C>(sh, q, rho, lane == 0, dw,
                                 initial_panels(q, static_cast<float>(rho),
                                                static_cast<float>(fabs(dw))),
                                 kMaxPanels, built, ok, lane, nodes);
    if (lane == 0) {
      out[i] = K;
      if (!ok) atomicAdd(bad, 1ULL);
    }
  }
}

// ---------------------------------------------------------------------------
// Radial interpolation mode (PHI_KERNEL_RADIAL)
// ---------------------------------------------------------------------------

// For one visibility, [GC](., dw) is an even function of rho band-limited to
// R cycles per grid pixel (the integral runs over r <= R).  radial_series
// integrates it by eval_chunk's quadrature at the Chebyshev points of pieces
// of [0, rho_max] of width L = 2 / R, and turns each piece's values into its
// Chebyshev coefficients in `ser` (in place); a piece whose two trailing
// coefficients exceed the tolerance is counted as unconverged.  radial_eval
// then gives the kernel at any rho <= rho_max by Clenshaw's recurrence.
template <typename T, typename C>
__device__ __forceinline__ int radial_series(C* ser, NodeVal<T>* sh, const QuadParams& q,
                                             const RadialView<T>& rv, T fu, T fv, int half,
                                             double dw, int lane, unsigned long long& my_bad,
                                             unsigned long long& my_nodes) {
  constexpr int NC = RadialN<T>::n;   // Chebyshev points per piece
  constexpr int NS = NC + 1;          // stride of a piece (offsets the banks)
  constexpr int PPW = 32 / NC;        // pieces transformed per warp pass
  const int max_pieces = rv.buf / NS;
  const float adw = static_cast<float>(fabs(dw));
  // farthest tap: |u offset| <= max(half - fu, fu + half - 1), likewise in v;
  // the piece count is clamped to the storage the plan sized for its
  // largest support (a rounding excess is extrapolated by the last piece)
  const T mu = fmax(static_cast<T>(half) - fu, fu + static_cast<T>(half - 1));
  const T mv = fmax(static_cast<T>(half) - fv, fv + static_cast<T>(half - 1));
  const T pf = ceil(sqrt(mu * mu + mv * mv) * rv.inv_L);
  int pieces = 1;
  if (pf >= static_cast<T>(max_pieces)) pieces = max_pieces;
  else if (pf > T(1)) pieces = static_cast<int>(pf);
  const int npts = pieces * NC;
  int built = 0;
  // the kernel at the Chebyshev points, 32 at a time in increasing rho
  for (int k0 = 0; k0 < npts; k0 += 32) {
    const int k = k0 + lane;
    const bool active = k < npts;
    const int kk = active ? k : npts - 1;   // idle lanes repeat the last point
    const int pc = kk / NC, j = kk - pc * NC;
    const T rho = rv.L * (static_cast<T>(pc) + rv.x1[j]);
    T rmax = rho;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    const int npan = initial_panels(q, static_cast<float>(rmax), adw);
    bool ok = true;
    const C K = eval_chunk<T, C>(sh, q, rho, active, dw, npan, kMaxPanels, built, ok, lane, my_nodes);
    if (active) {
      ser[pc * NS + j] = K;
      if (!ok) ++my_bad;
    }
  }
  __syncwarp();
  // c_m = (2 - [m == 0]) / NC sum_j f_j cos(pi m (j + 1/2) / NC), in place
  for (int p0 = 0; p0 < pieces; p0 += PPW) {
    const int pc = p0 + lane / NC, m = lane - (lane / NC) * NC;
    const bool on = lane < PPW * NC && pc < pieces;
    C c = cmake<C>(0.0, 0.0);
    if (on) {
      const C* f = ser + pc * NS;
      const T* dc = rv.dct + m;
#pragma unroll 4
      for (int j = 0; j < NC; ++j) {
        const T t = dc[j * NC];
        const C v = f[j];
        c.x = fma(v.x, t, c.x);
        c.y = fma(v.y, t, c.y);
      }
      const T sc = (m == 0 ? T(1) : T(2)) / static_cast<T>(NC);
      c.x *= sc;
      c.y *= sc;
    }
    __syncwarp();
    if (on) ser[pc * NS + m] = c;
    __syncwarp();
  }
  for (int pc = lane; pc < pieces; pc += 32) {
    const C* c = ser + pc * NS;
    T cmax = 0;
    for (int m = 0; m < NC; ++m) cmax = fmax(cmax, est_sqrt(c[m].x * c[m].x + c[m].y * c[m].y));
    const T tail = est_sqrt(c[NC - 1].x * c[NC - 1].x + c[NC - 1].y * c[NC - 1].y) +
                   est_sqrt(c[NC - 2].x * c[NC - 2].x + c[NC - 2].y * c[NC - 2].y);
    if (!(tail <= fmax(static_cast<T>(q.tol_abs), static_cast<T>(q.tol_rel) * cmax))) ++my_bad;
  }
  return pieces;
}

template <typename T, typename C>
__device__ __forceinline__ C radial_eval(const C* ser, const RadialView<T>& rv, int last, T last_f,
                                         T rho) {
  constexpr int NC = RadialN<T>::n;
  constexpr int NS = NC + 1;
  int ip;
  T fr;
  table_index(rho * rv.inv_L, last, last_f, ip, fr);
  const T x = fma(T(2), fr, T(-1));
  const T x2 = x + x;
  const C* c = ser + ip * NS;
  // Clenshaw: b_m = 2 x b_{m+1} - b_{m+2} + c_m;  K = x b_1 - b_2 + c_0
  if constexpr (sizeof(T) == 4) {
    // real and imaginary parts side by side in paired FP32 operations (the
    // same correctly rounded adds and multiply-adds as the scalar form)
    const float2 xx = make_float2(x2, x2);
    float2 b1 = make_float2(0.f, 0.f), b2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = NC - 1; m >= 1; --m) {
      const float2 nb = __ffma2_rn(xx, b1, __fadd2_rn(c[m], make_float2(-b2.x, -b2.y)));
      b2 = b1;
      b1 = nb;
    }
    return __ffma2_rn(make_float2(x, x), b1, __fadd2_rn(c[0], make_float2(-b2.x, -b2.y)));
  } else {
    T b1x = 0, b1y = 0, b2x = 0, b2y = 0;
#pragma unroll
    for (int m = NC - 1; m >= 1; --m) {
      const C cm = c[m];
      const T nx = fma(x2, b1x, cm.x - b2x);
      const T ny = fma(x2, b1y, cm.y - b2y);
      b2x = b1x;
      b2y = b1y;
      b1x = nx;
      b1y = ny;
    }
    const C c0 = c[0];
    C K;
    K.x = fma(x, b1x, c0.x - b2x);
    K.y = fma(x, b1y, c0.y - b2y);
    return K;
  }
}

// The radial mode's fused kernel: the series of each visibility, then every
// tap evaluated from it.
template <typename T, typename C, bool kGrid>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) vis_radial_kernel(
    const VisRec<T>* __restrict__ recs, const uint32_t* __restrict__ perm, int64_t n,
    const C* __restrict__ grid_in, C* grid_out, const C* __restrict__ vis_in,
    C* __restrict__ vis_out, QuadParams q, RadialView<T> rv,
    const int32_t* __restrict__ stack_slot, unsigned long long* head,
    unsigned long long* stats, int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  C* ser = reinterpret_cast<C*>(smem_raw + (blockDim.x >> 5) * kNodeBatch * sizeof(NodeVal<T>)) +
           warp * rv.buf;
  unsigned long long my_bad = 0, my_taps = 0, my_nodes = 0;
  const int npad = q.npad;
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    const int Jw = r.jw;
    const int64_t gbase = static_cast<int64_t>(stack_slot[r.stack]) * npad * npad;
    const int half = Jw / 2;
    const T fu = r.fu, fv = r.fv;
    const uint32_t pm = perm[i];
    const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                       : cmake<C>(0.0, 0.0);
    const int pieces = radial_series<T, C>(ser, sh, q, rv, fu, fv, half, r.dw, lane, my_bad,
                                           my_nodes);
    // every tap from its piece's series; taps t = b Jw + a in raster order,
    // advanced by 32 per chunk without a division per tap
    C accv = cmake<C>(0.0, 0.0);
    const int ntap = Jw * Jw;
    int a = lane % Jw, b = lane / Jw;
    const int step_b = 32 / Jw, step_a = 32 % Jw;
    T du_ = fu - static_cast<T>(a - half + 1), dv_ = fv - static_cast<T>(b - half + 1);
    const T fstep_a = static_cast<T>(step_a), fstep_b = static_cast<T>(step_b);
    const T fJw = static_cast<T>(Jw);
    const int last = pieces - 1;
    const T last_f = static_cast<T>(last);
    for (int t0 = 0; t0 < ntap; t0 += 32) {
      const int t = t0 + lane;
      if (t < ntap) {
        const int ou = a - half + 1, ov = b - half + 1;
        const C K = radial_eval<T, C>(ser, rv, last, last_f, sqrt(du_ * du_ + dv_ * dv_));
        const int64_t gi = gbase + static_cast<int64_t>(wrap_index(r.bv + ov, npad)) * npad +
                           wrap_index(r.bu + ou, npad);
        apply_tap<C, kGrid>(K, gi, yv, grid_in, grid_out, q.fx, accv);
      }
      a += step_a;
      b += step_b;
      du_ -= fstep_a;
      dv_ -= fstep_b;
      if (a >= Jw) {
        a -= Jw;
        ++b;
        du_ += fJw;
        dv_ -= T(1);
      }
    }
    // the series storage is rewritten by the next visibility's samples
    __syncwarp();
    if (lane == 0) my_taps += static_cast<unsigned long long>(ntap);
    if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
  }
  flush_counts(stats, my_bad, my_taps, my_nodes, lane);
}

// Direction-dependent effects (Sec. 5.2): vis_dde_kernel
#include "dde_kernel.cuh"

// ---------------------------------------------------------------------------
// Host side of the operator
// ---------------------------------------------------------------------------
namespace {

constexpr int kVisThreads = 256;

template <typename T, typename C>
int blocks_for_vis(const Plan& p, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vis_kernel<T, C, false>,
                                                    VisLaunch<T>::threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm * p.num_sms;
}

template <typename T, typename C>
size_t radial_smem(const Plan& p) {
  return (kVisThreads / 32) *
         (kNodeBatch * sizeof(NodeVal<T>) + static_cast<size_t>(p.radial_buf) * sizeof(C));
}

template <typename T, typename C>
RadialView<T> radial_view(const Plan& p) {
  RadialView<T> v;
  v.L = static_cast<T>(p.radial_L);
  v.inv_L = static_cast<T>(1.0 / p.radial_L);
  v.x1 = static_cast<const T*>(p.radial_tab);
  v.dct = static_cast<const T*>(p.radial_tab) + RadialN<T>::n;
  v.buf = p.radial_buf;
  return v;
}

// Chebyshev tables of the radial mode in the plan's precision, the piece
// width L = 2 / R and the series storage per warp for the largest support
// (every tap of a J_w box lies within sqrt(2) J_w / 2 of the visibility).
template <typename T, typename C>
int build_radial_tables_t(Plan& p, cudaStream_t s) {
  constexpr int n = RadialN<T>::n;
  std::vector<T> tab(n + n * n);
  for (int j = 0; j < n; ++j) {
    const double th = kPi * (j + 0.5) / n;
    tab[j] = static_cast<T>(0.5 * (1.0 + std::cos(th)));
    for (int m = 0; m < n; ++m) tab[n + j * n + m] = static_cast<T>(std::cos(m * th));
  }
  p.radial_L = 2.0 / p.R;
  const double rmax = std::sqrt(2.0) * std::max(p.max_jw, p.d.support) / 2.0;
  const int pieces = std::max(1, static_cast<int>(std::ceil(rmax / p.radial_L)));
  p.radial_buf = pieces * (n + 1);
  int dev = 0, optin = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (radial_smem<T, C>(p) > static_cast<size_t>(optin)) return PHI_ERR_SUPPORT;
  void* raw = nullptr;
  PHI_CUDA_TRY(cudaMalloc(&raw, sizeof(T) * tab.size()));
  p.radial_tab = raw;
  p.device_bytes += static_cast<int64_t>(sizeof(T) * tab.size());
  PHI_CUDA_TRY(cudaMemcpyAsync(p.radial_tab, tab.data(), sizeof(T) * tab.size(),
                               cudaMemcpyHostToDevice, s));
  PHI_CUDA_TRY(cudaStreamSynchronize(s));
  return PHI_OK;
}

template <typename T, typename C>
int build_table_t(Plan& p, cudaStream_t s) {
  const int64_t nr = p.table_nr, nw = p.table_nw;
  C* raw = nullptr;
  PHI_CUDA_TRY(cudaMalloc(&raw, sizeof(C) * nr * nw));
  const size_t smem = (kVisThreads / 32) * kNodeBatch * sizeof(NodeVal<T>);
  const int64_t want = (nw + 7) / 8;
  const int blocks = static_cast<int>(want < 65535 ? want : 65535);
  table_sample_kernel<T, C><<<blocks, kVisThreads, smem, s>>>(raw, nr, nw, p.table_hr, p.table_hw,
                                                              p.quad());
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    table_pair_kernel<C><<<p.num_sms * 8, 256, 0, s>>>(raw, nr, nw,
                                                       static_cast<KPair<C>*>(p.table));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(raw);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return PHI_ERR_CUDA;
  }
  return PHI_OK;
}

template <typename T, typename C>
TableView<T> table_view(const Plan& p) {
  TableView<T> v;
  v.pairs = p.table;
  v.nr = p.table_nr;
  v.nw = p.table_nw;
  v.inv_hr = static_cast<T>(1.0 / p.table_hr);
  v.inv_hw = static_cast<T>(1.0 / p.table_hw);
  v.fx.cells = p.fx_cells;
  v.fx.exp = p.fx_exp;
  return v;
}

// Visibilities a warp claims per queue atomic: about 1/32 of each warp's
// share, so the queue head is not contended when visibilities are cheap and
// the tail stays short when they are expensive.
inline int queue_batch(int64_t n, int64_t warps) {
  const int64_t b = n / (32 * (warps > 0 ? warps : 1));
  return static_cast<int>(b < 1 ? 1 : (b > 64 ? 64 : b));
}

#define PHI_TRY_ST(expr)        \
  do {                          \
    int st_ = (expr);           \
    if (st_ != PHI_OK) return st_; \
  } while (0)

// One launch over the uv-tile work items of stack k (items hold absolute
// record ranges; each item finds its stack's grid in the group by its key).
template <typename T, typename C, bool kGrid>
int launch_tile_table(Plan& p, int k, const C* grids_in, C* grids_out, const C* vis_in,
                      C* vis_out, cudaStream_t s) {
  const int64_t i0 = p.stack_item_off[k], ni = p.stack_item_off[k + 1] - i0;
  if (ni == 0) return PHI_OK;
  const int jmax = std::max(p.stack_jw[k], 2);
  const int side = p.tile + jmax;
  const size_t smem = sizeof(C) * static_cast<size_t>(side) * side;
  int dev = 0, optin = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  PHI_CUDA_TRY(cudaFuncGetAttributes(&fa, tile_table_kernel<T, C, kGrid>));
  if (smem + fa.sharedSizeBytes > static_cast<size_t>(optin)) {
    // the patch does not fit a block: this stack's records unstaged
    const int64_t b0 = p.stack_off[k], nk = p.stack_off[k + 1] - b0;
    const int blocks = p.num_sms * 8;
    vis_table_kernel<T, C, kGrid><<<blocks, kVisThreads, 0, s>>>(
        static_cast<const VisRec<T>*>(p.recs) + b0, p.perm + b0, nk, grids_in, grids_out, vis_in,
        vis_out, table_view<T, C>(p), p.npad, p.stack_slot_dev, p.counters + k, p.counters + p.K,
        queue_batch(nk, blocks * (kVisThreads / 32)));
    PHI_CUDA_TRY(cudaGetLastError());
    return PHI_OK;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_table_kernel<T, C, kGrid>,
                                                    kVisThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t want = static_cast<int64_t>(per_sm) * p.num_sms;
  const int blocks = static_cast<int>(ni < want ? ni : want);
  tile_table_kernel<T, C, kGrid><<<blocks, kVisThreads, smem, s>>>(
      static_cast<const VisRec<T>*>(p.recs), p.perm, p.item_start + 2 * i0, p.item_key + i0,
      static_cast<int>(ni), grids_in, grids_out, vis_in, vis_out, table_view<T, C>(p), p.npad,
      p.tile, p.tiles_per_row, jmax, p.stack_slot_dev, p.counters + k, p.counters + p.K);
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}

// One launch over the w-row work items of the group's stacks (grid_staging
// 2).  Sets `launched` to false (and launches nothing) when one row of the
// table does not fit a thread block's shared memory; the caller then runs
// the unstaged kernel.
template <typename T, typename C, bool kGrid>
int launch_row_table(Plan& p, int g, const C* grids_in, C* grids_out, const C* vis_in,
                     C* vis_out, cudaStream_t s, bool& launched) {
  launched = false;
  const int64_t s0 = p.group_off[g], s1 = p.group_off[g + 1];
  const int64_t i0 = p.stack_item_off[p.group_stacks[s0]];
  const int64_t ni = p.stack_item_off[p.group_stacks[s1 - 1] + 1] - i0;
  const size_t smem = sizeof(KPair<C>) * static_cast<size_t>(p.table_nr);
  int dev = 0, optin = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa;
  PHI_CUDA_TRY(cudaFuncGetAttributes(&fa, row_table_kernel<T, C, kGrid>));
  if (smem + fa.sharedSizeBytes > static_cast<size_t>(optin)) return PHI_OK;
  launched = true;
  if (ni == 0) return PHI_OK;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, row_table_kernel<T, C, kGrid>,
                                                    kVisThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t want = static_cast<int64_t>(per_sm) * p.num_sms;
  const int blocks = static_cast<int>(ni < want ? ni : want);
  row_table_kernel<T, C, kGrid><<<blocks, kVisThreads, smem, s>>>(
      static_cast<const VisRec<T>*>(p.recs), p.perm, p.row_idx, p.item_start + 2 * i0,
      p.item_key + i0, static_cast<int>(ni), grids_in, grids_out, vis_in, vis_out,
      table_view<T, C>(p), p.npad, p.stack_slot_dev, p.counters + g, p.counters + p.K);
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}

// In-place FFTs of the first n grids of the group (one batched call when
// the group is full).
template <typename T, typename C>
int fft_group(Plan& p, C* grids, int n, int dir, cudaStream_t s) {
  const int64_t plane = static_cast<int64_t>(p.npad) * p.npad;
  auto run = [&](cufftHandle h, C* g) -> cufftResult {
    if (cufftSetStream(h, s) != CUFFT_SUCCESS) return CUFFT_EXEC_FAILED;
    if (sizeof(T) == 8)
      return cufftExecZ2Z(h, reinterpret_cast<cufftDoubleComplex*>(g),
                          reinterpret_cast<cufftDoubleComplex*>(g), dir);
    return cufftExecC2C(h, reinterpret_cast<cufftComplex*>(g), reinterpret_cast<cufftComplex*>(g),
                        dir);
  };
  if (n == p.group && p.fft_batch_ok) {
    if (run(p.fft_batch, grids) != CUFFT_SUCCESS) return PHI_ERR_CUDA;
  } else {
    for (int i = 0; i < n; ++i)
      if (run(p.fft, grids + i * plane) != CUFFT_SUCCESS) return PHI_ERR_CUDA;
  }
  return PHI_OK;
}

// The fused kernel over all records of the group's stacks (contiguous in
// the sorted order).
// Per-visibility separable DDE kernels of phi_degrid_dde / phi_grid_dde.
struct DdeArgs {
  const void* a;
  const void* b;
  int jd;
};

// dde_warp_smem, launch_dde
#include "dde_launch.cuh"

template <typename T, typename C, bool kGrid>
int launch_group_kernel(Plan& p, int g, const C* grids_in, C* grids_out, const C* vis_in,
                        C* vis_out, cudaStream_t s, const DdeArgs* dde = nullptr) {
  const int64_t s0 = p.group_off[g], s1 = p.group_off[g + 1];
  if (dde) {
    const int64_t b0 = p.stack_off[p.group_stacks[s0]];
    const int64_t nk = p.stack_off[p.group_stacks[s1 - 1] + 1] - b0;
    if (nk == 0) return PHI_OK;
    return launch_dde<T, C, kGrid>(p, static_cast<const VisRec<T>*>(p.recs) + b0, b0, nk, g,
                                   grids_in, grids_out, vis_in, vis_out, *dde, s);
  }
  if (p.d.kernel_mode == PHI_KERNEL_TABLE && p.d.grid_staging == 2) {
    bool launched = false;
    PHI_TRY_ST((launch_row_table<T, C, kGrid>(p, g, grids_in, grids_out, vis_in, vis_out, s,
                                              launched)));
    if (launched) return PHI_OK;
  }
  if (p.d.kernel_mode == PHI_KERNEL_TABLE && p.d.grid_staging == 1) {
    for (int64_t i = s0; i < s1; ++i)
      PHI_TRY_ST((launch_tile_table<T, C, kGrid>(p, p.group_stacks[i], grids_in, grids_out, vis_in,
                                                 vis_out, s)));
    return PHI_OK;
  }
  const int64_t b0 = p.stack_off[p.group_stacks[s0]];
  const int64_t nk = p.stack_off[p.group_stacks[s1 - 1] + 1] - b0;
  if (nk == 0) return PHI_OK;
  const VisRec<T>* recs = static_cast<const VisRec<T>*>(p.recs) + b0;
  if (p.d.kernel_mode == PHI_KERNEL_RADIAL) {
    const size_t smem = radial_smem<T, C>(p);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vis_radial_kernel<T, C, kGrid>,
                                                      kVisThreads, smem) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const int blocks = per_sm * p.num_sms;
    vis_radial_kernel<T, C, kGrid><<<blocks, kVisThreads, smem, s>>>(
        recs, p.perm + b0, nk, grids_in, grids_out, vis_in, vis_out, p.quad(),
        radial_view<T, C>(p), p.stack_slot_dev, p.counters + g, p.counters + p.K,
        queue_batch(nk, blocks * (kVisThreads / 32)));
  } else if (p.d.kernel_mode == PHI_KERNEL_TABLE) {
    const int blocks = p.num_sms * 8;
    vis_table_kernel<T, C, kGrid><<<blocks, kVisThreads, 0, s>>>(
        recs, p.perm + b0, nk, grids_in, grids_out, vis_in, vis_out, table_view<T, C>(p), p.npad,
        p.stack_slot_dev, p.counters + g, p.counters + p.K,
        queue_batch(nk, blocks * (kVisThreads / 32)));
  } else {
    constexpr int threads = VisLaunch<T>::threads;
    const size_t smem = (threads / 32) * kNodeBatch * sizeof(NodeVal<T>);
    const int blocks = blocks_for_vis<T, C>(p, smem);
    vis_kernel<T, C, kGrid><<<blocks, threads, smem, s>>>(
        recs, p.perm + b0, nk, grids_in, grids_out, vis_in, vis_out, p.quad(), p.stack_slot_dev,
        p.counters + g, p.counters + p.K, queue_batch(nk, blocks * (threads / 32)));
  }
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}

template <typename T, typename C>
int run_degrid(Plan& p, const T* x, C* y, cudaStream_t s, const DdeArgs* dde = nullptr) {
  long ev = timer_begin(p, s);
  PHI_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(C) * (size_t)p.M, s));
  PHI_CUDA_TRY(cudaMemsetAsync(p.counters, 0, sizeof(unsigned long long) * p.K, s));
  timer_end(p, ev, PHI_STAGE_CLEAR, s);
  C* grids = static_cast<C*>(p.grid);
  const int ngroups = static_cast<int>(p.group_off.size()) - 1;
  for (int g = 0; g < ngroups; ++g) {
    const int n = static_cast<int>(p.group_off[g + 1] - p.group_off[g]);
    ev = timer_begin(p, s);
    prep_kernel<T, C><<<dim3(p.num_sms * 4, n), 256, 0, s>>>(
        x, p.omn_pix, static_cast<const T*>(p.corr_pix), p.N, p.npad, p.wbar_dev,
        p.group_stacks_dev + p.group_off[g], grids);
    PHI_CUDA_TRY(cudaGetLastError());
    timer_end(p, ev, PHI_STAGE_PREP, s);
    ev = timer_begin(p, s);
    PHI_TRY_ST((fft_group<T, C>(p, grids, n, CUFFT_FORWARD, s)));
    timer_end(p, ev, PHI_STAGE_FFT, s);
    ev = timer_begin(p, s);
    PHI_TRY_ST((launch_group_kernel<T, C, false>(p, g, grids, nullptr, nullptr, y, s, dde)));
    timer_end(p, ev, PHI_STAGE_DEGRID, s);
  }
  return PHI_OK;
}

// Deterministic plans, before a group's gridding: zero its fixed-point sums
// and set the exponent e from the call's largest term.  A cell receives at
// most one term per visibility and period of the grid its box covers, each
// at most |[GC]| times the visibility's factor; the bound on |[GC]| carries
// a factor 4 for the radial mode's Chebyshev interpolation (its Lebesgue
// constant is below 3 at 16 and 24 points) and the FP32 J0's rounding.
template <typename T, typename C>
int fixed_prepare(Plan& p, int g, const C* y, const DdeArgs* dde, cudaStream_t s) {
  const int64_t plane = static_cast<int64_t>(p.npad) * p.npad;
  const int n = static_cast<int>(p.group_off[g + 1] - p.group_off[g]);
  PHI_CUDA_TRY(cudaMemsetAsync(p.fx_cells, 0, 2 * sizeof(long long) * plane * n, s));
  PHI_CUDA_TRY(cudaMemsetAsync(p.fx_max, 0, sizeof(unsigned long long), s));
  const int64_t b0 = p.stack_off[p.group_stacks[p.group_off[g]]];
  const int64_t nk = p.stack_off[p.group_stacks[p.group_off[g + 1] - 1] + 1] - b0;
  if (nk > 0) {
    const int blocks = static_cast<int>(std::min<int64_t>(p.num_sms * 4, (nk + 255) / 256));
    fixed_bound_kernel<T, C><<<blocks, 256, 0, s>>>(
        static_cast<const VisRec<T>*>(p.recs) + b0, p.perm + b0, nk, y,
        dde ? static_cast<const C*>(dde->a) : nullptr,
        dde ? static_cast<const C*>(dde->b) : nullptr, dde ? dde->jd : 0, p.fx_max);
    PHI_CUDA_TRY(cudaGetLastError());
  }
  const int jbox = std::max(p.max_jw, 2) + (dde ? dde->jd - 1 : 0);
  const double periods = std::ceil(static_cast<double>(jbox) / p.npad);
  const double scale = 4.0 * p.kernel_bound * static_cast<double>(std::max<int64_t>(nk, 1)) *
                       periods * periods;
  // FP32 grids: 2^(32 - e) below FLT_MAX and 2^-e not below the smallest
  // subnormal; FP64 likewise for doubles
  const bool f64 = sizeof(T) == 8;
  fixed_exp_kernel<<<1, 1, 0, s>>>(p.fx_max, scale, f64 ? -990 : -95, f64 ? 1070 : 149,
                                   p.fx_exp);
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}

template <typename T, typename C>
int run_grid(Plan& p, const C* y, T* x, cudaStream_t s, const DdeArgs* dde = nullptr) {
  PHI_CUDA_TRY(cudaMemsetAsync(p.counters, 0, sizeof(unsigned long long) * p.K, s));
  C* grids = static_cast<C*>(p.grid);
  const int64_t plane = static_cast<int64_t>(p.npad) * p.npad;
  const int ngroups = static_cast<int>(p.group_off.size()) - 1;
  const bool fixed = p.fx_cells != nullptr;
  for (int g = 0; g < ngroups; ++g) {
    const int n = static_cast<int>(p.group_off[g + 1] - p.group_off[g]);
    long ev = timer_begin(p, s);
    if (fixed)
      PHI_TRY_ST((fixed_prepare<T, C>(p, g, y, dde, s)));
    else
      PHI_CUDA_TRY(cudaMemsetAsync(grids, 0, sizeof(C) * plane * n, s));
    timer_end(p, ev, PHI_STAGE_CLEAR, s);
    ev = timer_begin(p, s);
    PHI_TRY_ST((launch_group_kernel<T, C, true>(p, g, nullptr, grids, y, nullptr, s, dde)));
    if (fixed) {
      fixed_to_grid_kernel<T, C><<<p.num_sms * 8, 256, 0, s>>>(
          reinterpret_cast<const longlong2*>(p.fx_cells), p.fx_exp, plane * n, grids);
      PHI_CUDA_TRY(cudaGetLastError());
    }
    timer_end(p, ev, PHI_STAGE_GRID, s);
    ev = timer_begin(p, s);
    PHI_TRY_ST((fft_group<T, C>(p, grids, n, CUFFT_INVERSE, s)));
    timer_end(p, ev, PHI_STAGE_FFT, s);
    ev = timer_begin(p, s);
    finish_kernel<T, C><<<p.num_sms * 4, 256, 0, s>>>(
        grids, p.omn_pix, static_cast<const T*>(p.corr_pix), p.N, p.npad, p.wbar_dev,
        p.group_stacks_dev + p.group_off[g], n, x, g == 0 ? 0 : 1);
    PHI_CUDA_TRY(cudaGetLastError());
    timer_end(p, ev, PHI_STAGE_FINISH, s);
  }
  if (ngroups == 0) PHI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(T) * (size_t)p.N * p.N, s));
  return PHI_OK;
}

template <typename T, typename C>
int run_wkernel(Plan& p, const double* rho, const double* dw, int64_t n, C* out,
                int64_t* n_bad, cudaStream_t s) {
  unsigned long long* bad = p.counters + p.K + 2;
  PHI_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
  if (n > 0) {
    const size_t smem = (kVisThreads / 32) * kNodeBatch * sizeof(NodeVal<T>);
    int64_t want = (n + 7) / 8;
    int blocks = static_cast<int>(want < 65535 ? want : 65535);
    wkernel_kernel<T, C><<<blocks, kVisThreads, smem, s>>>(rho, dw, n, out, p.quad(), bad);
    PHI_CUDA_TRY(cudaGetLastError());
  }
  if (n_bad) {
    unsigned long long h = 0;
    PHI_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
    *n_bad = static_cast<int64_t>(h);
  }
  return PHI_OK;
}

}  // namespace

int build_kernel_table(Plan& p, cudaStream_t s) {
  if (p.d.precision == PHI_F64) return build_table_t<double, double2>(p, s);
  return build_table_t<float, float2>(p, s);
}

int build_radial_tables(Plan& p, cudaStream_t s) {
  if (p.d.precision == PHI_F64) return build_radial_tables_t<double, double2>(p, s);
  return build_radial_tables_t<float, float2>(p, s);
}

int compute_kernel_bound(Plan& p, double* scratch, cudaStream_t s) {
  const int blocks = (kMaxPanels + 127) / 128;
  if (p.d.precision == PHI_F64)
    kernel_bound_kernel<double><<<blocks, 128, 0, s>>>(static_cast<const double*>(p.node_hk),
                                                       scratch);
  else
    kernel_bound_kernel<float><<<blocks, 128, 0, s>>>(static_cast<const float*>(p.node_hk),
                                                      scratch);
  PHI_CUDA_TRY(cudaGetLastError());
  std::vector<double> h(kMaxPanels);
  PHI_CUDA_TRY(cudaMemcpyAsync(h.data(), scratch, sizeof(double) * kMaxPanels,
                               cudaMemcpyDeviceToHost, s));
  PHI_CUDA_TRY(cudaStreamSynchronize(s));
  p.kernel_bound = *std::max_element(h.begin(), h.end());
  return PHI_OK;
}

long timer_begin(Plan& p, cudaStream_t s) {
  if (!p.timing) return -1;
  size_t idx = 2 * p.ev_pending.size();
  while (p.ev_pool.size() < idx + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    p.ev_pool.push_back(e);
  }
  if (cudaEventRecord(p.ev_pool[idx], s) != cudaSuccess) return -1;
  return static_cast<long>(idx);
}

void timer_end(Plan& p, long idx, int stage, cudaStream_t s) {
  if (idx < 0) return;
  if (cudaEventRecord(p.ev_pool[idx + 1], s) != cudaSuccess) return;
  p.ev_pending.emplace_back(stage, static_cast<size_t>(idx));
}

template <typename T, typename C>
cudaError_t set_dde_smem(int bytes) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(vis_dde_kernel<T, C, false, false>, a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(vis_dde_kernel<T, C, true, false>, a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(vis_dde_kernel<T, C, false, true>, a, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(vis_dde_kernel<T, C, true, true>, a, bytes);
  return e;
}

// The largest dynamic shared memory a block of `kernel` may use: the opt-in
// limit less the kernel's static shared memory.
template <typename K>
cudaError_t set_max_dynamic_smem(K kernel, int optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - static_cast<int>(fa.sharedSizeBytes));
}

template <typename T, typename C>
cudaError_t set_staging_smem(int optin) {
  cudaError_t e = set_max_dynamic_smem(tile_table_kernel<T, C, false>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(tile_table_kernel<T, C, true>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(row_table_kernel<T, C, false>, optin);
  if (e == cudaSuccess) e = set_max_dynamic_smem(row_table_kernel<T, C, true>, optin);
  return e;
}

int set_kernel_smem_limits() {
  const size_t f32 = (kVisThreads / 32) * kNodeBatch * sizeof(NodeVal<float>);
  const size_t f64 = (kVisThreads / 32) * kNodeBatch * sizeof(NodeVal<double>);
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_kernel<float, float2, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_kernel<float, float2, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32));
  PHI_CUDA_TRY(cudaFuncSetAttribute(wkernel_kernel<float, float2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_kernel<double, double2, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_kernel<double, double2, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64));
  PHI_CUDA_TRY(cudaFuncSetAttribute(wkernel_kernel<double, double2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64));
  PHI_CUDA_TRY(cudaFuncSetAttribute(table_sample_kernel<float, float2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32));
  PHI_CUDA_TRY(cudaFuncSetAttribute(table_sample_kernel<double, double2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64));
  // radial mode: its series storage depends on the plan; allow up to the
  // device's opt-in limit (plans that would need more are refused)
  int dev = 0, optin = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_radial_kernel<float, float2, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_radial_kernel<float, float2, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_radial_kernel<double, double2, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  PHI_CUDA_TRY(cudaFuncSetAttribute(vis_radial_kernel<double, double2, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  PHI_CUDA_TRY((set_dde_smem<float, float2>(optin)));
  PHI_CUDA_TRY((set_dde_smem<double, double2>(optin)));
  // table staging: patch and row sizes depend on the plan; the attribute is
  // process-wide, so plans used from several threads at once all set the
  // same value, the opt-in limit (larger patches and rows fall back to the
  // unstaged kernel)
  PHI_CUDA_TRY((set_staging_smem<float, float2>(optin)));
  PHI_CUDA_TRY((set_staging_smem<double, double2>(optin)));
  return PHI_OK;
}

}  // namespace phi

extern "C" int phi_degrid(phi_plan_t plan, const void* image_dev, void* vis_dev, void* stream) {
  if (!plan || (!image_dev && plan->M > 0) || (!vis_dev && plan->M > 0)) return PHI_ERR_ARG;
  phi::Plan& p = *plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.M == 0) return PHI_OK;
  if (p.d.precision == PHI_F64)
    return phi::run_degrid<double, double2>(p, static_cast<const double*>(image_dev),
                                            static_cast<double2*>(vis_dev), s);
  return phi::run_degrid<float, float2>(p, static_cast<const float*>(image_dev),
                                        static_cast<float2*>(vis_dev), s);
}

extern "C" int phi_grid(phi_plan_t plan, const void* vis_dev, void* image_dev, void* stream) {
  if (!plan || !image_dev || (!vis_dev && plan->M > 0)) return PHI_ERR_ARG;
  phi::Plan& p = *plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.d.precision == PHI_F64)
    return phi::run_grid<double, double2>(p, static_cast<const double2*>(vis_dev),
                                          static_cast<double*>(image_dev), s);
  return phi::run_grid<float, float2>(p, static_cast<const float2*>(vis_dev),
                                      static_cast<float*>(image_dev), s);
}

namespace {
int dde_check(phi_plan_t plan, const void* a, const void* b, int32_t taps) {
  if (!plan || taps < 1 || taps > 15 || taps % 2 == 0) return PHI_ERR_ARG;
  if (plan->M > 0 && (!a || !b)) return PHI_ERR_ARG;
  if (plan->d.conj_fold) return PHI_ERR_ARG;
  return PHI_OK;
}
}  // namespace

extern "C" int phi_degrid_dde(phi_plan_t plan, const void* image_dev, const void* dde_a_dev,
                              const void* dde_b_dev, int32_t dde_taps, void* vis_dev,
                              void* stream) {
  const int st = dde_check(plan, dde_a_dev, dde_b_dev, dde_taps);
  if (st != PHI_OK) return st;
  if ((!image_dev || !vis_dev) && plan->M > 0) return PHI_ERR_ARG;
  phi::Plan& p = *plan;
  if (p.M == 0) return PHI_OK;
  const phi::DdeArgs dde{dde_a_dev, dde_b_dev, dde_taps};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.d.precision == PHI_F64)
    return phi::run_degrid<double, double2>(p, static_cast<const double*>(image_dev),
                                            static_cast<double2*>(vis_dev), s, &dde);
  return phi::run_degrid<float, float2>(p, static_cast<const float*>(image_dev),
                                        static_cast<float2*>(vis_dev), s, &dde);
}

extern "C" int phi_grid_dde(phi_plan_t plan, const void* vis_dev, const void* dde_a_dev,
                            const void* dde_b_dev, int32_t dde_taps, void* image_dev,
                            void* stream) {
  const int st = dde_check(plan, dde_a_dev, dde_b_dev, dde_taps);
  if (st != PHI_OK) return st;
  if (!image_dev || (!vis_dev && plan->M > 0)) return PHI_ERR_ARG;
  phi::Plan& p = *plan;
  const phi::DdeArgs dde{dde_a_dev, dde_b_dev, dde_taps};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p.d.precision == PHI_F64)
    return phi::run_grid<double, double2>(p, static_cast<const double2*>(vis_dev),
                                          static_cast<double*>(image_dev), s, &dde);
  return phi::run_grid<float, float2>(p, static_cast<const float2*>(vis_dev),
                                      static_cast<float*>(image_dev), s, &dde);
}

extern "C" int phi_wkernel(phi_plan_t plan, const double* rho_dev, const double* dw_dev, int64_t n,
                           void* k_dev, int64_t* n_unconverged, void* stream) {
  if (!plan || n < 0 || (n > 0 && (!rho_dev || !dw_dev || !k_dev))) return PHI_ERR_ARG;
  phi::Plan& p = *plan;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_unconverged) PHI_TRY_NOT_CAPTURING(s);
  if (p.d.precision == PHI_F64)
    return phi::run_wkernel<double, double2>(p, rho_dev, dw_dev, n, static_cast<double2*>(k_dev),
                                             n_unconverged, s);
  return phi::run_wkernel<float, float2>(p, rho_dev, dw_dev, n, static_cast<float2*>(k_dev),
                                         n_unconverged, s);
}

extern "C" int phi_plan_set_timing(phi_plan_t plan, int enable) {
  if (!plan) return PHI_ERR_ARG;
  plan->timing = enable != 0;
  return PHI_OK;
}

extern "C" int phi_plan_timings(phi_plan_t plan, double* ms, int64_t* launches, int reset,
                                void* stream) {
  if (!plan) return PHI_ERR_ARG;
  phi::Plan& p = *plan;
  PHI_CUDA_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  for (const auto& pr : p.ev_pending) {
    float t = 0.f;
    PHI_CUDA_TRY(cudaEventSynchronize(p.ev_pool[pr.second + 1]));
    PHI_CUDA_TRY(cudaEventElapsedTime(&t, p.ev_pool[pr.second], p.ev_pool[pr.second + 1]));
    p.stage_ms[pr.first] += t;
    p.stage_launches[pr.first] += 1;
  }
  p.ev_pending.clear();
  for (int i = 0; i < PHI_NUM_STAGES; ++i) {
    if (ms) ms[i] = p.stage_ms[i];
    if (launches) launches[i] = p.stage_launches[i];
    if (reset) {
      p.stage_ms[i] = 0.0;
      p.stage_launches[i] = 0;
    }
  }
  return PHI_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free kernel evaluation (phi_wkernel_noalloc)
//
// Callers that cannot allocate device memory while running get the plan-free
// evaluator below.  Its scratch -- node tables for panel counts 1..64 and the
// unconverged counter -- is this file-scope array rather than plan memory.
// The array's name is only a host-side stand-in for the device object; the
// kernels receive the device address that cudaGetSymbolAddress returns.
// ---------------------------------------------------------------------------
namespace phi {
namespace {

constexpr int kNoAllocMaxPanels = PHI_WKERNEL_NOALLOC_MAX_PANELS;
constexpr int64_t kNoAllocNodes =
    static_cast<int64_t>(kNodes) * kNoAllocMaxPanels * (kNoAllocMaxPanels + 1) / 2;
constexpr size_t kNoAllocBytes = PHI_WKERNEL_NOALLOC_SCRATCH_BYTES;
static_assert(kNoAllocBytes == 256 + 3 * 8 * kNoAllocNodes, "scratch layout");

// [0, 256): counter; then omn (FP64), hk, hd (8 bytes per node reserved each).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device).
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return PHI_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      (void)cudaGetLastError();
      return PHI_ERR_CUDA;
    }
    g_noalloc_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return PHI_OK;
}

template <typename T, typename C>
__global__ void __launch_bounds__(256) wkernel_noalloc_kernel(const double* __restrict__ rho_in,
                                                              const double* __restrict__ dw_in,
                                                              int64_t n, C* __restrict__ out,
                                                              QuadParams q, int max_panels,
                                                              unsigned long long* bad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = blockIdx.x * wpb + warp; i < n; i += (int64_t)gridDim.x * wpb) {
    const T rho = static_cast<T>(rho_in[i]);
    const double dw = dw_in[i];
    int built = 0;
    bool ok = true;
    unsigned long long nodes = 0;
    const C K = eval_chunk<T, C>(
        sh, q, rho, lane == 0, dw,
        initial_panels(q, static_cast<float>(rho), static_cast<float>(fabs(dw))), max_panels,
        built, ok, lane, nodes);
    if (lane == 0) {
      out[i] = K;
      if (!ok) atomicAdd(bad, 1ULL);
    }
  }
}

template <typename T, typename C>
int run_wkernel_noalloc(const phi_wkernel_params& prm, const double* rho, const double* dw,
                        int64_t n, C* out, int64_t* n_bad, cudaStream_t s) {
  unsigned char* base = nullptr;
  int st = noalloc_scratch(&base);
  if (st != PHI_OK) return st;
  const size_t smem = (kVisThreads / 32) * kNodeBatch * sizeof(NodeVal<T>);
  PHI_CUDA_TRY(cudaFuncSetAttribute(wkernel_noalloc_kernel<T, C>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(base);
  double* omn = reinterpret_cast<double*>(base + 256);
  T* hk = reinterpret_cast<T*>(base + 256 + 8 * kNoAllocNodes);
  T* hd = reinterpret_cast<T*>(base + 256 + 16 * kNoAllocNodes);
  const int64_t nodes = panel_table_offset(prm.max_panels + 1);
  const double l_win = prm.window_radius / prm.du;
  const double n_win = sqrt(1.0 - l_win * l_win);
  QuadParams q;
  q.R = prm.window_radius;
  q.Rf = static_cast<float>(prm.window_radius);
  q.chirp_coeff = static_cast<float>(l_win / (n_win * prm.du));
  q.inv_cycles = static_cast<float>(1.0 / prm.cycles_per_panel);
  q.tol_rel = static_cast<float>(prm.quad_rel_tol);
  q.tol_abs = static_cast<float>(prm.quad_abs_tol);
  q.max_refine = prm.max_refine;
  q.npad = 0;
  q.node_omn = omn;
  q.node_hk = hk;
  q.node_hd = hd;
  q.tap_order = nullptr;
  q.tap_off = nullptr;
  // the counter keeps the previous call's value: clear it first
  PHI_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s));
  node_table_kernel<T><<<static_cast<int>((nodes + 255) / 256), 256, 0, s>>>(
      prm.window_radius, prm.du, 0.5 * prm.support, prm.kb_beta, omn, hk, hd, nodes);
  PHI_CUDA_TRY(cudaGetLastError());
  if (n > 0) {
    const int64_t want = (n + 7) / 8;
    const int blocks = static_cast<int>(want < 65535 ? want : 65535);
    wkernel_noalloc_kernel<T, C><<<blocks, kVisThreads, smem, s>>>(rho, dw, n, out, q,
                                                                   prm.max_panels, bad);
    PHI_CUDA_TRY(cudaGetLastError());
  }
  if (n_bad) {
    unsigned long long h = 0;
    PHI_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, s));
    PHI_CUDA_TRY(cudaStreamSynchronize(s));
    *n_bad = static_cast<int64_t>(h);
  }
  return PHI_OK;
}

}  // namespace
}  // namespace phi

extern "C" int phi_wkernel_noalloc(const phi_wkernel_params* params, const double* rho_dev,
                                   const double* dw_dev, int64_t n, void* k_dev,
                                   int64_t* n_unconverged, void* stream) {
  if (!params || n < 0 || (n > 0 && (!rho_dev || !dw_dev || !k_dev))) return PHI_ERR_ARG;
  const phi_wkernel_params& p = *params;
  if (p.max_panels < 1 || p.max_panels > PHI_WKERNEL_NOALLOC_MAX_PANELS) return PHI_ERR_ARG;
  if (p.support < 2 || p.support > 64 || p.support % 2) return PHI_ERR_ARG;
  if (!(p.du > 0.0) || !(p.window_radius > 0.0) || !(p.kb_beta > 0.0)) return PHI_ERR_ARG;
  if (!(p.quad_rel_tol > 0.0) || !(p.quad_abs_tol > 0.0) || !(p.cycles_per_panel > 0.0))
    return PHI_ERR_ARG;
  if (p.max_refine < 0 || p.max_refine > 8) return PHI_ERR_ARG;
  if (p.precision != PHI_F32 && p.precision != PHI_F64) return PHI_ERR_ARG;
  if (p.window_radius / p.du >= 1.0) return PHI_ERR_HORIZON;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_unconverged) PHI_TRY_NOT_CAPTURING(s);
  if (p.precision == PHI_F64)
    return phi::run_wkernel_noalloc<double, double2>(p, rho_dev, dw_dev, n,
                                                     static_cast<double2*>(k_dev), n_unconverged, s);
  return phi::run_wkernel_noalloc<float, float2>(p, rho_dev, dw_dev, n,
                                                 static_cast<float2*>(k_dev), n_unconverged, s);
}
