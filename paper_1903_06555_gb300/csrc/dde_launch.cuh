// Host launcher of vis_dde_kernel.  Not a standalone header: phi_ops.cu
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
  if (warps < 1) return PHI_ERR_SUPPORT;
  const size_t smem = per_warp * warps;
  const bool radial = p.d.kernel_mode == PHI_KERNEL_RADIAL;
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
