// Launch-side view of the kernels: per-(lattice, storage) shapes and the
// host launchers that the engine dispatches to.  Each storage type's kernels
// are compiled in their own translation unit (step_<type>.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "step_kernel.cuh"

namespace lbm {

// CTA width, TMA pipeline depth and the CTAs per SM the register budget is
// sized for, per (lattice, storage).  Shared memory per CTA is
// NS * (Q box slots + flag slot) + the psi ring.
// (Measured on GB300, 8192x4096: D2Q9 NS 4 / MINB 8 for FP32 and MINB 10 for
// 16-bit storage beat NS 5 / MINB 6 and MINB 8 or 12 (16-bit at MINB 12: 76
// registers, 0.243 ms against 0.233); D2Q21 needs NS >= R + 2 = 5, and NS 5
// with 3 CTAs per SM (FP32) or 5 (16-bit) beat NS 6 with 2 or 3 by 21% and
// 5%.  16-bit D2Q21 runs CTAs of 64 threads (node pairs), its plane groups
// arriving as boxes of depth 1, 3 and 7: NS 6 (43 KB, 5 CTAs per SM: two rows
// in flight besides the four the collision re-reads) beat NS 5 (6 CTAs) by 1.1%
// and NS 7 (4 CTAs) by 8%.)
template <int Q, typename S> struct StepConfig {
  static constexpr int W = 128;
  static constexpr int NS = (Q == 9) ? (sizeof(S) == 8 ? 4 : (sizeof(S) == 4 ? 4 : 5))
                                     : (sizeof(S) == 2 ? 6 : 5);
  static constexpr int MINB = (Q == 9) ? (sizeof(S) == 8 ? 2 : (sizeof(S) == 4 ? 8 : 10))
                                       : (sizeof(S) == 8 ? 1 : (sizeof(S) == 4 ? 3 : 6));
  // The persistent batch kernel carries its tile loop on top of the march:
  // 16-bit D2Q9 targets 8 CTAs per SM there, so that it does not spill.
  static constexpr int BATCH_MINB = (Q == 9 && sizeof(S) == 2) ? 8 : MINB;
  // One CTA per tile, the compile-time-flag kernel (kFlExpPlain): D2Q9 FP32
  // and 16-bit batches run 12 CTAs per SM (76-80 registers, no spills; the
  // 256-lattice sweep 6% faster than at 10 for FP16S, 1.4% than at 8 for
  // FP32): short tiles of many small lattices need more CTAs in flight than
  // the single lattice's long strips.  The run-time-flag kernel keeps MINB (it
  // would spill at 12).
  static constexpr int BATCH_MINB_PLAIN = (Q == 9 && sizeof(S) != 8) ? 12 : MINB;
  template <int FL> static constexpr int batch_minb_tile() {
    return FL == kFlExpPlain ? BATCH_MINB_PLAIN : MINB;
  }
};

template <int Q, typename S>
using ConfigShape = StepShape<Q, S, StepConfig<Q, S>::W, StepConfig<Q, S>::NS>;

// Launches the fused step (mode kModeStep) or the read-out pass (kModeMoments).
template <int Q, typename S>
cudaError_t launch_step(const PopMaps& src, const CUtensorMap& flags,
                        const StepArgs<typename Codec<S>::T, S>& a, dim3 grid,
                        cudaStream_t stream, int mode);

// CTAs of the step kernel that fit on one SM (occupancy query).
template <int Q, typename S> int step_ctas_per_sm();

// One time step of up to BatchArgs::kChunk members of a batch: nctas CTAs, one per
// tile of the chunk, or (persistent) each marching every nctas-th tile; and
// the batch kernel's residency per SM.  `plain`: every member has the
// exponential psi, no projection and (16-bit storage) stochastic rounding, so
// the kernel with those settings fixed runs.
template <int Q, typename S>
cudaError_t launch_batch(const BatchArgs<typename Codec<S>::T, S>& args,
                         const BatchMember<typename Codec<S>::T, S>* members, int nctas,
                         int parity, bool persistent, bool plain, cudaStream_t stream);
template <int Q, typename S> int batch_ctas_per_sm();

// Auxiliary kernels (aux.cu).
template <int Q, typename S>
cudaError_t launch_encode(const double* f, S* buf, int nx, int ny, int64_t pitch, int64_t plane,
                          double rho_s, cudaStream_t st);
template <int Q, typename S>
cudaError_t launch_equilibrium(const double* rho, const double* ux, const double* uy,
                               const double* dfi, S* buf, int nx, int ny, int64_t pitch,
                               int64_t plane, double rho_s, cudaStream_t st);
template <int Q, typename S>
cudaError_t launch_decode(const S* buf, double* f, int nx, int ny, int64_t pitch, int64_t plane,
                          double rho_s, cudaStream_t st);
template <int Q, typename T>
cudaError_t launch_wall_prepare(const double* phi, const double* psr, const double* psa,
                                const double* uw, double G_R, double G_A, double eps, int nx,
                                int ny, T* phie, T* sx, T* sy, T* uwx, T* uwy, uint32_t* flags,
                                int nchunk_pad, cudaStream_t st);

// Compensated (Neumaier) FP64 sums of up to three [N] arrays (NULL sums to
// 0) into out[3]: nparts blocks each reduce a grid-stride share into
// partials[6 * nparts], then one thread merges them in block order
// (deterministic).  lbm_totals and lbm_reduce3_noalloc both use kReduceParts
// blocks.
constexpr int kReduceParts = 1024;
cudaError_t launch_reduce3(const double* a, const double* b, const double* c, int64_t n,
                           double* partials, int nparts, double* out, cudaStream_t st);
cudaError_t launch_colsum(const double* f, int q, int64_t n, double* out_n, cudaStream_t st);

cudaError_t launch_filter_pass(int q, const double* g, double* out, const uint8_t* solid, int nx,
                               int ny, cudaStream_t st);

}  // namespace lbm
