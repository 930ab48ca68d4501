// The DDE convolution kernel (Sec. 5.2), vis_dde_kernel.  Not a standalone
// header: phi_ops.cu includes it inside namespace phi, after the quadrature,
// tap and work-queue pieces it uses, so that it is compiled with them in one
// translation unit while its source stays apart from the other kernels'.
#pragma once

// ---------------------------------------------------------------------------
// Direction-dependent effects (Sec. 5.2)
// ---------------------------------------------------------------------------

// W-kernel rows per band of vis_dde_kernel in radial mode.
constexpr int kDdeBand = 8;

// Elements (of the complex type) of one warp's DDE storage beside its node
// buffer, then the two DDE kernels and, in radial mode, the visibility's
// series.  Quadrature: the whole J_max x J_max w-kernel box (its taps are
// integrated in ring order, whose chunks group taps of similar radius).
// Radial mode (banded): a band of w-kernel rows (kDdeBand x J_max) and the
// ring of row-pass rows (kDdeBand + J_D - 1 rows of J_max + J_D - 1).
__host__ __device__ inline int dde_warp_elems(int jmax, int jd, int ser, bool banded) {
  return (banded ? kDdeBand * jmax + (kDdeBand + jd - 1) * (jmax + jd - 1) : jmax * jmax) +
         2 * jd + ser;
}

// The separable convolution's two passes over one row pass value and one
// combined tap: a complex multiply-add.
template <typename C>
__device__ __forceinline__ void cmad(C& acc, const C& a, const C& b) {
  acc.x += a.x * b.x - a.y * b.y;
  acc.y += a.x * b.y + a.y * b.x;
}

// Degrid / grid with a separable DDE kernel D_i(s) = a_i(s_u) b_i(s_v)
// (J_D = 2 h + 1 taps a side, caller's visibility order) convolved with the
// w-kernel: with a_s, b_s the kernels' entries s = 0 .. J_D - 1 (offset
// s - h) and K the J_w x J_w w-kernel box, every tap of the
// (J_w + J_D - 1)^2 box is C(cv, cu) = sum_s b_s R(cv - 2 h + s, cu), from
// the row pass R(kb, cu) = sum_s a_s K(kb, cu - 2 h + s) (terms outside the
// box left out), i.e. C(q) = sum_s D(s) [GC](u - q - s): J_D J_w (2 J_w +
// J_D - 1) complex multiply-adds per visibility instead of J_D^2 + J_D per
// combined tap.  One warp per visibility.
//
// Quadrature: the warp integrates the whole box (ring order, kVisTaps taps
// per lane, as vis_kernel) into shared memory; each lane then takes one
// column cu and a run of rows, forming each row of R once, when its walk
// reaches it, into slot kb mod J_D of the lane's own column of a ring kept
// in the node buffer (free by then), and summing J_D of them per combined
// tap.  Blocks of fewer than 32 columns split their rows into runs so that
// every lane works.
//
// Radial mode: the taps come cheaply from the visibility's series, so the
// warp walks the box in bands of kDdeBand rows instead, which stores only a
// band and leaves room for more warps per SM: it evaluates a band's taps,
// forms those rows of R into a ring of kDdeBand + 2 h rows (row kb in ring
// row kb mod (kDdeBand + 2 h), so the 2 h rows of the band above stay
// readable) and emits the combined rows the ring now completes: cv in
// [k0, k1), and [J_w, J_w + 2 h) after the last band.  (Banding the
// quadrature path too ran 18% slower: chunks confined to a band group
// radii less well and fill fewer lanes.)
template <typename T, typename C, bool kGrid, bool kRadial>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) vis_dde_kernel(
    const VisRec<T>* __restrict__ recs, const uint32_t* __restrict__ perm, int64_t n,
    const C* __restrict__ grid_in, C* grid_out, const C* __restrict__ vis_in,
    C* __restrict__ vis_out, QuadParams q, RadialView<T> rv, const C* __restrict__ dde_a,
    const C* __restrict__ dde_b, int jd, int jmax, const int32_t* __restrict__ stack_slot,
    unsigned long long* head, unsigned long long* stats, int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int h = jd >> 1;
  const int nring = kDdeBand + 2 * h;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  // quadrature: the box; radial: the band, then the ring of R rows
  C* box = reinterpret_cast<C*>(smem_raw + (blockDim.x >> 5) * kNodeBatch * sizeof(NodeVal<T>)) +
           warp * dde_warp_elems(jmax, jd, kRadial ? rv.buf : 0, kRadial);
  C* ring = kRadial ? box + kDdeBand * jmax : reinterpret_cast<C*>(sh);
  C* dab = kRadial ? ring + nring * (jmax + 2 * h) : box + jmax * jmax;   // a_i then b_i
  C* ser = dab + 2 * jd;                                                  // the series
  static_assert(32 * 15 * sizeof(C) <= kNodeBatch * sizeof(NodeVal<T>),
                "the per-lane ring of the largest DDE kernel must fit the node buffer");
  unsigned long long my_bad = 0, my_taps = 0, my_nodes = 0;
  const int npad = q.npad;
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    const int Jw = r.jw, Jc = Jw + 2 * h;
    const int64_t gbase = static_cast<int64_t>(stack_slot[r.stack]) * npad * npad;
    const int half = Jw / 2;
    const T fu = r.fu, fv = r.fv;
    const uint32_t pm = perm[i];
    const int64_t src = pm & 0x7fffffffu;
    const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                       : cmake<C>(0.0, 0.0);
    if (lane < 2 * jd) dab[lane] = lane < jd ? dde_a[src * jd + lane] : dde_b[src * jd + lane - jd];
    C accv = cmake<C>(0.0, 0.0);
    // one combined tap from its rows of R: row kb at rows[(kb mod nmod) stride]
    auto emit = [&](int cv, int cu, const C* rows, int stride, int nmod) {
      const int lo = max(0, cv - 2 * h), hi = min(Jw - 1, cv);
      C acc = cmake<C>(0.0, 0.0);
      for (int kb = lo, sl = lo % nmod; kb <= hi; ++kb, sl = sl + 1 == nmod ? 0 : sl + 1)
        cmad(acc, dab[jd + kb - cv + 2 * h], rows[sl * stride]);
      ++my_taps;
      const int ou = cu - h - half + 1, ov = cv - h - half + 1;
      const int64_t gi = gbase + static_cast<int64_t>(wrap_index(r.bv + ov, npad)) * npad +
                         wrap_index(r.bu + ou, npad);
      apply_tap<C, kGrid>(acc, gi, yv, grid_in, grid_out, q.fx, accv);
    };
    if constexpr (kRadial) {
      const int last =
          radial_series<T, C>(ser, sh, q, rv, fu, fv, half, r.dw, lane, my_bad, my_nodes) - 1;
      const T last_f = static_cast<T>(last);
      for (int k0 = 0; k0 < Jw; k0 += kDdeBand) {
        const int k1 = min(Jw, k0 + kDdeBand), nrow = k1 - k0;
        // 1. w-kernel rows [k0, k1) into the band
        for (int t = lane; t < nrow * Jw; t += 32) {
          const int rr = t / Jw, ka = t - rr * Jw;
          const T du_ = fu - static_cast<T>(ka - half + 1);
          const T dv_ = fv - static_cast<T>(k0 + rr - half + 1);
          box[t] = radial_eval<T, C>(ser, rv, last, last_f, sqrt(du_ * du_ + dv_ * dv_));
        }
        __syncwarp();
        // 2. row pass of the band's rows into ring rows kb mod nring
        for (int e = lane; e < nrow * Jc; e += 32) {
          const int rr = e / Jc, cu = e - rr * Jc;
          C acc = cmake<C>(0.0, 0.0);
          for (int s = 0; s < jd; ++s) {
            const int ka = cu - 2 * h + s;
            if (ka >= 0 && ka < Jw) cmad(acc, dab[s], box[rr * Jw + ka]);
          }
          ring[((k0 + rr) % nring) * Jc + cu] = acc;
        }
        __syncwarp();
        // 3. the combined rows the ring now completes
        const int c1 = k1 == Jw ? Jc : k1;
        for (int e = lane; e < (c1 - k0) * Jc; e += 32) {
          const int dv = e / Jc, cu = e - dv * Jc;
          emit(k0 + dv, cu, ring + cu, Jc, nring);
        }
        // the band and the ring rows are rewritten by the next band
        __syncwarp();
      }
    } else {
      // 1. the w-kernel box by the per-tap quadrature, ring order
      const uint16_t* order = q.tap_order + q.tap_off[half - 1];
      const float adw = static_cast<float>(fabs(r.dw));
      const int ntap = Jw * Jw;
      int built = 0;
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
        eval_chunk_nt<kVisTaps>(sh, q, rho, act, r.dw, npan, kMaxPanels, built, ok, lane,
                                my_nodes, K);
#pragma unroll
        for (int k = 0; k < kVisTaps; ++k)
          if (act[k]) {
            box[(code[k] >> 8) * Jw + (code[k] & 0xffu)] = K[k];
            if (!ok[k]) ++my_bad;
          }
      }
      __syncwarp();
      // 2. per lane: one column, a run of rows, the lane's ring column
      for (int c0 = 0; c0 < Jc; c0 += 32) {
        const int nb = min(32, Jc - c0);
        const int runs = 32 / nb, len = (Jc + runs - 1) / runs;
        const int run = lane / nb, cu = c0 + lane - run * nb;
        const int r0 = run * len, r1 = min(Jc, r0 + len);
        if (run >= runs || r0 >= r1) continue;
        C* ring_l = ring + lane;
        // row kb of R at column cu into slot kb mod jd (`slot`, advanced
        // with the walk)
        int slot = max(0, r0 - 2 * h) % jd;
        auto row_pass = [&](int kb) {
          C acc = cmake<C>(0.0, 0.0);
          for (int s = 0; s < jd; ++s) {
            const int ka = cu - 2 * h + s;
            if (ka >= 0 && ka < Jw) cmad(acc, dab[s], box[kb * Jw + ka]);
          }
          ring_l[slot * 32] = acc;
          slot = slot + 1 == jd ? 0 : slot + 1;
        };
        for (int kb = max(0, r0 - 2 * h); kb < min(r0, Jw); ++kb) row_pass(kb);
        for (int cv = r0; cv < r1; ++cv) {
          if (cv < Jw) row_pass(cv);
          emit(cv, cu, ring_l, 32, jd);
        }
      }
    }
    // the box, the DDE taps and the ring are rewritten for the next visibility
    __syncwarp();
    if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
  }
  flush_counts(stats, my_bad, my_taps, my_nodes, lane);
}

// Two-pass DDE convolution.  A whole w-kernel box in shared memory (11.5 KB
// at J_w = 38), or a band of it with its ring, leaves room for few warps per
// SM, which starves the quadrature of the latency hiding it needs, so when
// that happens the box goes through global memory instead: dde_box_kernel
// (or dde_box_radial_kernel in radial mode) computes the boxes of a chunk of
// visibilities with the plain kernel's warp layout and occupancy, and
// dde_conv_kernel forms their combined taps with the separable passes and
// applies them, holding only the DDE kernels and the row-pass ring in
// shared memory.

// Pass 1: the J_w x J_w w-kernel box of each of records [0, n) into
// boxes[i * jmax^2], row-major with row length J_w.
template <typename T, typename C>
__global__ void __launch_bounds__(VisLaunch<T>::threads, VisLaunch<T>::min_blocks)
    dde_box_kernel(const VisRec<T>* __restrict__ recs, int64_t n, C* __restrict__ boxes,
                   int jmax, QuadParams q, unsigned long long* head,
                   unsigned long long* stats, int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  unsigned long long my_bad = 0, my_nodes = 0;
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    const int Jw = r.jw, half = Jw / 2, ntap = Jw * Jw;
    C* box = boxes + static_cast<int64_t>(i) * jmax * jmax;
    const T fu = r.fu, fv = r.fv;
    const uint16_t* order = q.tap_order + q.tap_off[half - 1];
    const float adw = static_cast<float>(fabs(r.dw));
    int built = 0;
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
          box[(code[k] >> 8) * Jw + (code[k] & 0xffu)] = K[k];
          if (!ok[k]) ++my_bad;
        }
    }
  }
  // unconverged taps and tap-node evaluations into the statistics (the taps
  // themselves are counted by pass 2, as combined taps)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_bad += __shfl_xor_sync(0xffffffffu, my_bad, o);
    my_nodes += __shfl_xor_sync(0xffffffffu, my_nodes, o);
  }
  if (lane == 0) {
    if (my_bad) atomicAdd(stats, my_bad);
    if (my_nodes) atomicAdd(stats + 3, my_nodes);
  }
}

// Pass 1 in radial mode: each visibility's series (radial_series, with
// vis_radial_kernel's block shape: node buffers, then a series buffer per
// warp), then its box from the series, row-major with row length J_w.
template <typename T, typename C>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) dde_box_radial_kernel(
    const VisRec<T>* __restrict__ recs, int64_t n, C* __restrict__ boxes, int jmax, QuadParams q,
    RadialView<T> rv, unsigned long long* head, unsigned long long* stats, int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  NodeVal<T>* sh = reinterpret_cast<NodeVal<T>*>(smem_raw) + warp * kNodeBatch;
  C* ser = reinterpret_cast<C*>(smem_raw + (blockDim.x >> 5) * kNodeBatch * sizeof(NodeVal<T>)) +
           warp * rv.buf;
  unsigned long long my_bad = 0, my_nodes = 0;
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    const int Jw = r.jw, half = Jw / 2, ntap = Jw * Jw;
    C* box = boxes + static_cast<int64_t>(i) * jmax * jmax;
    const T fu = r.fu, fv = r.fv;
    const int last =
        radial_series<T, C>(ser, sh, q, rv, fu, fv, half, r.dw, lane, my_bad, my_nodes) - 1;
    const T last_f = static_cast<T>(last);
    for (int t = lane; t < ntap; t += 32) {
      const int kb = t / Jw, ka = t - kb * Jw;
      const T du_ = fu - static_cast<T>(ka - half + 1);
      const T dv_ = fv - static_cast<T>(kb - half + 1);
      box[t] = radial_eval<T, C>(ser, rv, last, last_f, sqrt(du_ * du_ + dv_ * dv_));
    }
    // the series is rewritten for the next visibility
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_bad += __shfl_xor_sync(0xffffffffu, my_bad, o);
    my_nodes += __shfl_xor_sync(0xffffffffu, my_nodes, o);
  }
  if (lane == 0) {
    if (my_bad) atomicAdd(stats, my_bad);
    if (my_nodes) atomicAdd(stats + 3, my_nodes);
  }
}

// Pass 2: records [0, n) with their boxes from pass 1; the combined taps by
// the separable passes, each lane one column and a run of rows with its
// ring column in shared memory (jd x 32 per warp, after the warp's DDE
// kernels).  A lane's grid column is fixed for its run and its grid row
// advances by one per combined row, so neither is wrapped per tap.
template <typename T, typename C, bool kGrid>
__global__ void __launch_bounds__(256) dde_conv_kernel(
    const VisRec<T>* __restrict__ recs, const uint32_t* __restrict__ perm, int64_t n,
    const C* __restrict__ boxes, int jmax, const C* __restrict__ grid_in, C* grid_out,
    const C* __restrict__ vis_in, C* __restrict__ vis_out, const C* __restrict__ dde_a,
    const C* __restrict__ dde_b, int jd, int npad, FixedGrid fx,
    const int32_t* __restrict__ stack_slot, unsigned long long* head,
    unsigned long long* stats, int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  C* dab = reinterpret_cast<C*>(smem_raw) + warp * (2 * jd + 32 * jd);   // a_i then b_i
  C* ring_l = dab + 2 * jd + lane;                                       // this lane's column
  const C* dbv = dab + jd;
  const int h = jd >> 1, h2 = 2 * h;
  unsigned long long my_taps = 0;
  WarpQueue wq;
  unsigned long long i;
  while (wq.take(head, static_cast<unsigned long long>(batch), n, lane, i)) {
    const VisRec<T> r = recs[i];
    const int Jw = r.jw, Jc = Jw + h2, half = Jw / 2;
    const C* __restrict__ box = boxes + static_cast<int64_t>(i) * jmax * jmax;
    // the row walk reads the box a row at a time: ask L2 for all of it now
    // (addresses inside the box only; a prefetch is a hint and loads nothing)
    {
      const char* bp = reinterpret_cast<const char*>(box);
      const int nbytes = Jw * Jw * static_cast<int>(sizeof(C));
      for (int off = lane * 128; off < nbytes; off += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(bp + off));
    }
    const int64_t gbase = static_cast<int64_t>(stack_slot[r.stack]) * npad * npad;
    const uint32_t pm = perm[i];
    const int64_t src = pm & 0x7fffffffu;
    const C yv = kGrid ? load_visibility<T, C>(vis_in, pm, static_cast<T>(r.weight))
                       : cmake<C>(0.0, 0.0);
    if (lane < 2 * jd) dab[lane] = lane < jd ? dde_a[src * jd + lane] : dde_b[src * jd + lane - jd];
    __syncwarp();
    C accv = cmake<C>(0.0, 0.0);
    for (int c0 = 0; c0 < Jc; c0 += 32) {
      const int nb = min(32, Jc - c0);
      const int runs = 32 / nb, len = (Jc + runs - 1) / runs;
      const int run = lane / nb, cu = c0 + lane - run * nb;
      const int r0 = run * len, r1 = min(Jc, r0 + len);
      if (run >= runs || r0 >= r1) continue;
      // the row pass's taps of this column: box columns cu - 2 h + s, s in [s0, s1)
      const int s0 = max(0, h2 - cu), s1 = min(jd, Jw + h2 - cu);
      const int ka0 = cu - h2;   // box column of s = 0
      const int64_t gcol = gbase + wrap_index(r.bu + cu - h - half + 1, npad);
      int grow = wrap_index(r.bv + r0 - h - half + 1, npad);
      // rows of R from max(0, r0 - 2 h) on; row kb sits in ring slot kb mod jd
      int kb_next = max(0, r0 - h2);
      int slot = kb_next % jd;
      for (int cv = r0; cv < r1; ++cv) {
        for (; kb_next <= min(cv, Jw - 1); ++kb_next) {
          C acc = cmake<C>(0.0, 0.0);
          const int k0 = kb_next * Jw + ka0;   // k0 + s >= kb_next * Jw for s >= s0
          for (int s = s0; s < s1; ++s) cmad(acc, dab[s], box[k0 + s]);
          ring_l[slot * 32] = acc;
          slot = slot + 1 == jd ? 0 : slot + 1;
        }
        // rows kb = cv - 2 h .. cv of R inside the box, b index kb - cv + 2 h
        const int lo = max(0, cv - h2), hi = min(Jw - 1, cv);
        C acc = cmake<C>(0.0, 0.0);
        int sl = slot - (hi - lo + 1);
        if (sl < 0) sl += jd;
        for (int kb = lo, jb = lo - cv + h2; kb <= hi; ++kb, ++jb) {
          cmad(acc, dbv[jb], ring_l[sl * 32]);
          sl = sl + 1 == jd ? 0 : sl + 1;
        }
        ++my_taps;
        apply_tap<C, kGrid>(acc, gcol + static_cast<int64_t>(grow) * npad, yv, grid_in, grid_out,
                            fx, accv);
        grow = grow + 1 == npad ? 0 : grow + 1;
      }
    }
    // the DDE taps and the ring are rewritten for the next visibility
    __syncwarp();
    if (!kGrid) store_visibility<T, C>(accv, static_cast<T>(r.weight), pm, vis_out, lane);
  }
  flush_counts(stats, 0, my_taps, 0, lane);
}
