// Definitions of the step launchers; included by one translation unit per
// storage type, which instantiates them for D2Q9 and D2Q21.
#pragma once

#include "launch.cuh"

namespace lbm {

template <int Q, typename S, int MODE, int FL>
static cudaError_t prepare_kernel() {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  static cudaError_t once = cudaFuncSetAttribute(
      step_kernel<Q, S, Cfg::W, Cfg::NS, MODE, Cfg::MINB, FL>,
      cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  return once;
}

// The fused step as a programmatic dependent launch: the step may begin
// launching while the previous kernel in the stream drains (the kernel waits
// before touching global memory).
template <int Q, typename S, int FL>
static cudaError_t launch_step_pdl(const PopMaps& src, const CUtensorMap& flags,
                                   const StepArgs<typename Codec<S>::T, S>& a, dim3 grid,
                                   cudaStream_t stream) {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  cudaError_t e;
  if ((e = prepare_kernel<Q, S, kModeStep, FL>()) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(Sh::NT);
  cfg.dynamicSmemBytes = Sh::SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_kernel<Q, S, Cfg::W, Cfg::NS, kModeStep, Cfg::MINB, FL>,
                            src, flags, a);
}

template <int Q, typename S>
cudaError_t launch_step(const PopMaps& src, const CUtensorMap& flags,
                        const StepArgs<typename Codec<S>::T, S>& a, dim3 grid,
                        cudaStream_t stream, int mode) {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  cudaError_t e;
  if (mode == kModeStep) {
    // The common settings (exponential psi, no projection, stochastic
    // rounding of 16-bit storage) run a kernel with them fixed at compile time.
    const bool plain = a.phys.psi_kind == 0 && !a.phys.project &&
                       (a.stochastic || !Codec<S>::kShifted);
    e = plain ? launch_step_pdl<Q, S, kFlExpPlain>(src, flags, a, grid, stream)
              : launch_step_pdl<Q, S, kFlRuntime>(src, flags, a, grid, stream);
    if (e != cudaSuccess) return e;
  } else {
    if ((e = prepare_kernel<Q, S, kModeMoments, kFlRuntime>()) != cudaSuccess) return e;
    step_kernel<Q, S, Cfg::W, Cfg::NS, kModeMoments, Cfg::MINB, kFlRuntime>
        <<<grid, Sh::NT, Sh::SMEM, stream>>>(src, flags, a);
  }
  return cudaGetLastError();
}

template <int Q, typename S> int step_ctas_per_sm() {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  if (prepare_kernel<Q, S, kModeStep, kFlRuntime>() != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, step_kernel<Q, S, Cfg::W, Cfg::NS, kModeStep, Cfg::MINB, kFlRuntime>, Sh::NT,
          Sh::SMEM) != cudaSuccess)
    return 0;
  return n;
}

template <int Q, typename S, int FL>
static cudaError_t prepare_batch_kernel() {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  static cudaError_t once = [] {
    cudaError_t e = cudaFuncSetAttribute(
        batch_step_kernel<Q, S, Cfg::W, Cfg::NS, Cfg::template batch_minb_tile<FL>(), false, FL>,
        cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(batch_step_kernel<Q, S, Cfg::W, Cfg::NS, Cfg::BATCH_MINB, true, FL>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
  }();
  return once;
}

template <int Q, typename S, int FL>
static cudaError_t launch_batch_fl(const BatchArgs<typename Codec<S>::T, S>& args,
                                   const BatchMember<typename Codec<S>::T, S>* members,
                                   int nctas, int parity, bool persistent, cudaStream_t stream) {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  cudaError_t e = prepare_batch_kernel<Q, S, FL>();
  if (e != cudaSuccess) return e;
  // A programmatic dependent launch, as for the single-lattice step.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nctas);
  cfg.blockDim = dim3(Sh::NT);
  cfg.dynamicSmemBytes = Sh::SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (persistent)
    return cudaLaunchKernelEx(&cfg, batch_step_kernel<Q, S, Cfg::W, Cfg::NS, Cfg::BATCH_MINB, true, FL>,
                              args, members, parity);
  return cudaLaunchKernelEx(&cfg, batch_step_kernel<Q, S, Cfg::W, Cfg::NS, Cfg::template batch_minb_tile<FL>(), false, FL>,
                            args, members, parity);
}

template <int Q, typename S>
cudaError_t launch_batch(const BatchArgs<typename Codec<S>::T, S>& args,
                         const BatchMember<typename Codec<S>::T, S>* members, int nctas,
                         int parity, bool persistent, bool plain, cudaStream_t stream) {
  return plain ? launch_batch_fl<Q, S, kFlExpPlain>(args, members, nctas, parity, persistent, stream)
               : launch_batch_fl<Q, S, kFlRuntime>(args, members, nctas, parity, persistent, stream);
}

// Residency per SM of the persistent batch kernel; also sets the shared-memory
// attribute of every batch kernel variant (outside any stream capture).
template <int Q, typename S> int batch_ctas_per_sm() {
  using Cfg = StepConfig<Q, S>;
  using Sh = ConfigShape<Q, S>;
  if (prepare_batch_kernel<Q, S, kFlRuntime>() != cudaSuccess) return 0;
  if (prepare_batch_kernel<Q, S, kFlExpPlain>() != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &n, batch_step_kernel<Q, S, Cfg::W, Cfg::NS, Cfg::BATCH_MINB, true, kFlRuntime>, Sh::NT,
          Sh::SMEM) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace lbm

#define LBM_INSTANTIATE_STEP(Q, S)                                                         \
  template cudaError_t lbm::launch_step<Q, S>(const PopMaps&, const CUtensorMap&,      \
                                              const lbm::StepArgs<lbm::Codec<S>::T, S>&,   \
                                              dim3, cudaStream_t, int);                    \
  template int lbm::step_ctas_per_sm<Q, S>();                                            \
  template cudaError_t lbm::launch_batch<Q, S>(                                          \
      const lbm::BatchArgs<lbm::Codec<S>::T, S>&,                                         \
      const lbm::BatchMember<lbm::Codec<S>::T, S>*, int, int, bool, bool, cudaStream_t);    \
  template int lbm::batch_ctas_per_sm<Q, S>();
