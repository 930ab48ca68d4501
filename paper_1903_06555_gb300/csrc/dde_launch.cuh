// Host launchers of the DDE kernels.  Not a standalone header: phi_ops.cu
// includes it inside its host-side anonymous namespace, after DdeArgs,
// queue_batch and radial_view.
#pragma once

// Shared memory of one warp of vis_dde_kernel: the quadrature nodes, the
// w-kernel box (quadrature) or a band of it and the ring of row-pass rows
// (radial mode) for the plan's largest support, the two DDE kernels and, in
// radial mode, the series.
template <typename T, typename C>
size_t dde_warp_smem(const Plan& p, int jd) {
  const int jmax = std::max(p.max_jw, 2);
  const bool radial = p.d.kernel_mode == PHI_KERNEL_RADIAL;
  return kNodeBatch * sizeof(NodeVal<T>) +
         static_cast<size_t>(dde_warp_elems(jmax, jd, radial ? p.radial_buf : 0, radial)) *
             sizeof(C);
}

// Plans whose single-pass DDE kernel would keep fewer warps than this
// resident per SM take the two-pass path; its transient box buffer
// holds at most kDdeBoxBytes (chunks of visibilities otherwise).
constexpr int kDdeTwoPassWarps = 24;
constexpr size_t kDdeBoxBytes = size_t(2) << 30;

// The two-pass DDE convolution (dde_box_kernel, dde_conv_kernel) over
// records [b0, b0 + nk) of group g, through a stream-ordered buffer
// (cudaMallocAsync / cudaFreeAsync: no device-wide synchronisation).  Sets
// `launched` to false, launching nothing, when that buffer cannot be had.
template <typename T, typename C, bool kGrid>
int launch_dde_two_pass(Plan& p, const VisRec<T>* recs, int64_t b0, int64_t nk, int g,
                        const C* grids_in, C* grids_out, const C* vis_in, C* vis_out,
                        const DdeArgs& dde, cudaStream_t s, bool& launched) {
  launched = false;
  const int jmax = std::max(p.max_jw, 2);
  const size_t box_bytes = sizeof(C) * static_cast<size_t>(jmax) * jmax;
  const int64_t chunk =
      std::min<int64_t>(nk, std::max<int64_t>(1, static_cast<int64_t>(kDdeBoxBytes / box_bytes)));
  C* boxes = nullptr;
  const cudaError_t ea = cudaMallocAsync(reinterpret_cast<void**>(&boxes), box_bytes * chunk, s);
  if (ea == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    return PHI_OK;
  }
  PHI_CUDA_TRY(ea);
  launched = true;
  // pass 1: the plain kernel's block shape and shared memory (limits set
  // to one value for all plans, so concurrent launchers agree)
  const bool radial = p.d.kernel_mode == PHI_KERNEL_RADIAL;
  constexpr int box_threads = VisLaunch<T>::threads;
  const size_t box_smem = radial ? radial_smem<T, C>(p)
                                 : (box_threads / 32) * kNodeBatch * sizeof(NodeVal<T>);
  int dev = 0, optin = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (radial)
    PHI_CUDA_TRY(cudaFuncSetAttribute(dde_box_radial_kernel<T, C>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  else
    PHI_CUDA_TRY(cudaFuncSetAttribute(
        dde_box_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        static_cast<int>((box_threads / 32) * kNodeBatch * sizeof(NodeVal<T>))));
  int box_per_sm = 0, conv_per_sm = 0;
  const cudaError_t eo =
      radial ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   &box_per_sm, dde_box_radial_kernel<T, C>, box_threads, box_smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&box_per_sm, dde_box_kernel<T, C>,
                                                             box_threads, box_smem);
  if (eo != cudaSuccess || box_per_sm < 1) box_per_sm = 1;
  // pass 2: the DDE kernels (2 jd) and the ring (32 jd) per warp; the limit
  // is that of the largest jd (15), the same for every plan
  const size_t conv_smem = (kVisThreads / 32) * 34 * static_cast<size_t>(dde.jd) * sizeof(C);
  PHI_CUDA_TRY(cudaFuncSetAttribute(dde_conv_kernel<T, C, kGrid>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>((kVisThreads / 32) * 34 * 15 * sizeof(C))));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&conv_per_sm, dde_conv_kernel<T, C, kGrid>,
                                                    kVisThreads, conv_smem) != cudaSuccess ||
      conv_per_sm < 1)
    conv_per_sm = 1;
  const int box_blocks = box_per_sm * p.num_sms, conv_blocks = conv_per_sm * p.num_sms;
  unsigned long long* head = p.counters + g;
  int st = PHI_OK;
  for (int64_t c0 = 0; c0 < nk && st == PHI_OK; c0 += chunk) {
    const int64_t n = std::min(chunk, nk - c0);
    if (cudaMemsetAsync(head, 0, sizeof(unsigned long long), s) != cudaSuccess) {
      st = PHI_ERR_CUDA;
      break;
    }
    if (radial)
      dde_box_radial_kernel<T, C><<<box_blocks, box_threads, box_smem, s>>>(
          recs + c0, n, boxes, jmax, p.quad(), radial_view<T, C>(p), head, p.counters + p.K,
          queue_batch(n, box_blocks * (box_threads / 32)));
    else
      dde_box_kernel<T, C><<<box_blocks, box_threads, box_smem, s>>>(
          recs + c0, n, boxes, jmax, p.quad(), head, p.counters + p.K,
          queue_batch(n, box_blocks * (box_threads / 32)));
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemsetAsync(head, 0, sizeof(unsigned long long), s) != cudaSuccess) {
      st = PHI_ERR_CUDA;
      break;
    }
    dde_conv_kernel<T, C, kGrid><<<conv_blocks, kVisThreads, conv_smem, s>>>(
        recs + c0, p.perm + b0 + c0, n, boxes, jmax, grids_in, grids_out, vis_in, vis_out,
        static_cast<const C*>(dde.a), static_cast<const C*>(dde.b), dde.jd, p.npad, p.quad().fx,
        p.stack_slot_dev, head, p.counters + p.K, queue_batch(n, conv_blocks * (kVisThreads / 32)));
    if (cudaGetLastError() != cudaSuccess) st = PHI_ERR_CUDA;
  }
  const cudaError_t ef = cudaFreeAsync(boxes, s);
  if (st != PHI_OK) return st;
  PHI_CUDA_TRY(ef);
  return PHI_OK;
}

template <typename T, typename C, bool kGrid>
int launch_dde(Plan& p, const VisRec<T>* recs, int64_t b0, int64_t nk, int g, const C* grids_in,
               C* grids_out, const C* vis_in, C* vis_out, const DdeArgs& dde, cudaStream_t s) {
  int dev = 0, optin = 0, per_sm_smem = 0, reserved = 0;
  PHI_CUDA_TRY(cudaGetDevice(&dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                      dev));
  PHI_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  // warps per block that keep the most warps resident per SM (the boxes are
  // large: a block of 8 can leave most of an SM's shared memory unused)
  const size_t per_warp = dde_warp_smem<T, C>(p, dde.jd);
  int warps = 0, best = 0;
  for (int w = 1; w <= kVisThreads / 32; ++w) {
    const size_t blk = per_warp * w;
    if (blk > static_cast<size_t>(optin)) break;
    const int resident = w * static_cast<int>(per_sm_smem / (blk + reserved));
    if (resident >= best) {
      best = resident;
      warps = w;
    }
  }
  const bool radial = p.d.kernel_mode == PHI_KERNEL_RADIAL;
  if (best < kDdeTwoPassWarps) {
    bool launched = false;
    PHI_TRY_ST((launch_dde_two_pass<T, C, kGrid>(p, recs, b0, nk, g, grids_in, grids_out, vis_in,
                                                 vis_out, dde, s, launched)));
    if (launched) return PHI_OK;
  }
  if (warps < 1) return PHI_ERR_SUPPORT;
  const size_t smem = per_warp * warps;
  auto kernel = radial ? vis_dde_kernel<T, C, kGrid, true> : vis_dde_kernel<T, C, kGrid, false>;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * warps, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int blocks = per_sm * p.num_sms;
  const RadialView<T> rv = radial ? radial_view<T, C>(p) : RadialView<T>{};
  kernel<<<blocks, 32 * warps, smem, s>>>(
      recs, p.perm + b0, nk, grids_in, grids_out, vis_in, vis_out, p.quad(), rv,
      static_cast<const C*>(dde.a), static_cast<const C*>(dde.b), dde.jd, std::max(p.max_jw, 2),
      p.stack_slot_dev, p.counters + g, p.counters + p.K, queue_batch(nk, blocks * warps));
  PHI_CUDA_TRY(cudaGetLastError());
  return PHI_OK;
}
