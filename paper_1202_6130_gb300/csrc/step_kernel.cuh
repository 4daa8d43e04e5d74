// The fused time step: one kernel launch per step over every lattice node.
//
// Per node (Sec. II of arXiv:1202.6130): pull the Q populations (streaming),
// rho and j (Eqs. M0, M1), psi(rho), the fluid-fluid force (Eq. force_SC) from
// the neighbours' psi, the long-range fluid-solid force rho S and the wall
// momentum exchange rho phi^eps (U_wall - u - F_FF / rho) (Eqs. force_SC_FS,
// wall_shift), the optional projection, the EDM-BGK collision (Eq. BE-BGK),
// and the store of the post-collision populations.
//
// Layout.  Populations are structure-of-arrays [Q][ny + 2 GY][pitch] with GX
// ghost columns on each side of a row and GY ghost rows above and below; the
// ghosts hold periodic images, written by the step itself, so every pull is an
// in-bounds read and every TMA box starts on a 16-byte boundary.  The buffer
// holds post-collision values f_i^post(x) at the emitting node; the next step
// pulls f_i(x) = f_i^post(x - c_i).
//
// Schedule.  A CTA of W threads owns a strip of W columns and a segment of L
// rows, and marches down the segment one node row at a time.  Each row's Q
// source rows (one per population, shifted by -c_y) arrive by TMA into one of
// NS shared-memory stages, NS - R - 1 rows ahead of use.  psi is computed once
// per node (plus R halo nodes on each side of the strip) into a ring of 2R+1
// rows; the collision of row k - R then reads its neighbours' psi from the
// ring, so psi never touches HBM and the only redundant traffic is the 2R halo
// columns and rows of each strip segment.
#pragma once

#include <cuda.h>

#include "lattice.cuh"
#include "node.cuh"
#include "tma.cuh"

namespace lbm {

enum : uint32_t { kStatusNonFinite = 1u, kStatusTimeout = 2u };

enum StepMode : int {
  kModeStep = 0,      // write post-collision populations to fout
  kModeMoments = 1,   // write rho and u = (j + F/2) / rho (FP64) instead
};

template <typename T, typename S> struct StepArgs {
  Physics<T> phys;
  WallFields<T> wall;
  int32_t nx, ny;
  int32_t pitch;       // elements per padded row
  int32_t tile_rows;   // L
  int64_t plane;       // elements per population plane
  S* fout;             // kModeStep: destination buffer (same layout as the source)
  double* out_rho;     // kModeMoments: [ny][nx]
  double* out_ux;
  double* out_uy;
  int32_t momentum;    // kModeMoments: 1 -> out_ux/out_uy get j + F/2 instead of u
  uint32_t* status;    // error bits (kStatus*)
};

template <int Q, typename S, int W, int NS> struct StepShape {
  using L = Lattice<Q>;
  using T = typename Codec<S>::T;
  static constexpr int R = L::R;
  static constexpr int GX = ghost_x<S, R>();
  static constexpr int GY = ghost_y<R>();
  static constexpr int BW = W + 2 * GX;                                 // box width (elements)
  static constexpr int SLOT = ((BW * (int)sizeof(S) + 127) / 128) * 128;  // bytes per box
  static constexpr int SLOT_E = SLOT / (int)sizeof(S);
  static constexpr int STAGE = Q * SLOT;
  static constexpr int RING_W = W + 2 * R;
  static constexpr int RING_H = 2 * R + 1;
  static constexpr int SMEM = 128 /*alignment slack*/ + NS * STAGE + NS * 8 +
                              RING_H * RING_W * (int)sizeof(T) + 16;
  static constexpr uint32_t TX_BYTES = Q * BW * (uint32_t)sizeof(S);
};

template <int Q, typename S, int W, int NS, int MODE>
__global__ void __launch_bounds__(W)
    step_kernel(const __grid_constant__ CUtensorMap src, const StepArgs<typename Codec<S>::T, S> a) {
  using Sh = StepShape<Q, S, W, NS>;
  using L = Lattice<Q>;
  using T = typename Codec<S>::T;
  using C = Codec<S>;
  constexpr int R = Sh::R;
  constexpr int GX = Sh::GX;
  constexpr int GY = Sh::GY;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  unsigned char* stages = base;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + NS * Sh::STAGE);
  T* ring = reinterpret_cast<T*>(bars + NS);
  int* s_abort = reinterpret_cast<int*>(ring + Sh::RING_H * Sh::RING_W);

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * W;
  const int y0 = blockIdx.y * a.tile_rows;
  const int Lr = min(a.tile_rows, a.ny - y0);
  const int K = Lr + 2 * R;  // node rows y0 - R .. y0 + Lr + R - 1
  const int x = x0 + tid;

  uint64_t policy = 0;
  if (tid == 0) {
    prefetch_tensormap(&src);
#pragma unroll 1
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    *s_abort = 0;
    fence_barrier_init();
    policy = l2_policy_evict_first();
  }
  __syncthreads();

  // Thread 0 issues the Q boxes of node row k into stage k % NS.
  auto issue = [&](int k) {
    const int s = k % NS;
    const int ynode = y0 - R + k;
    mbar_arrive_expect_tx(&bars[s], Sh::TX_BYTES);
    unsigned char* st = stages + s * Sh::STAGE;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      tma_load_3d(st + i * Sh::SLOT, &src, &bars[s], x0, ynode - L::cy(i) + GY, i, policy);
    }
  };
  int issued = 0;
  if (tid == 0) {
    const int n0 = min(NS, K);
#pragma unroll 1
    for (int k = 0; k < n0; ++k) issue(k);
    issued = n0;
  }

  // Per-population decode shift w_i rho_s (zero unless shifted storage).
  const T rho_s = a.phys.rho_s;

  auto load_pop = [&](const S* st, int i, int xl) -> T {
    // xl: node column relative to x0; pulled from column xl - c_x in the box,
    // whose first element is node column -GX.
    return C::dec(st[i * Sh::SLOT_E + xl + GX - L::cx(i)], T(L::w(i)) * rho_s);
  };

  auto psi_at = [&](const S* st, int xl) -> T {
    T rho = load_pop(st, 0, xl);
#pragma unroll
    for (int i = 1; i < Q; ++i) rho += load_pop(st, i, xl);
    return pseudo_potential<Q, T>(a.phys, rho);
  };

  int k = 0;
#pragma unroll 1
  for (; k < K; ++k) {
    const int s = k % NS;
    if (!mbar_wait_bounded(&bars[s], (uint32_t)(k / NS) & 1u)) *s_abort = 1;
    const S* st = reinterpret_cast<const S*>(stages + s * Sh::STAGE);
    T* ring_row = ring + (k % Sh::RING_H) * Sh::RING_W;
    ring_row[tid + R] = psi_at(st, tid);
    if (tid < 2 * R) {
      const int xl = tid < R ? tid - R : W + tid - R;
      ring_row[xl + R] = psi_at(st, xl);
    }
    __syncthreads();
    if (*s_abort) break;

    if (k >= 2 * R) {
      const int ko = k - R;
      const int yo = y0 - R + ko;
      const S* sto = reinterpret_cast<const S*>(stages + (ko % NS) * Sh::STAGE);
      T f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = load_pop(sto, i, tid);
      T rho, jx, jy;
      node_moments<Q, T>(f, rho, jx, jy);
      const T inv_rho = T(1) / rho;
      const T ux = div_rho<T>(jx, rho, inv_rho);
      const T uy = div_rho<T>(jy, rho, inv_rho);

      // sum_i w_i psi(x + c_i) c_i from the ring (rest state contributes 0).
      const T psi_c = ring[(ko % Sh::RING_H) * Sh::RING_W + tid + R];
      T sfx = 0, sfy = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (L::cx(i) == 0 && L::cy(i) == 0) continue;
        const T nb = ring[((ko + L::cy(i)) % Sh::RING_H) * Sh::RING_W + tid + R + L::cx(i)];
        const T wn = T(L::w(i)) * nb;
        if (L::cx(i) != 0) sfx += wn * T(L::cx(i));
        if (L::cy(i) != 0) sfy += wn * T(L::cy(i));
      }

      // Wall terms: only where the per-(row, 32-column chunk) flag is set.
      bool has_wall = false;
      T phie = 0, Sx = 0, Sy = 0, uwx = 0, uwy = 0;
      if (a.wall.active && x < a.nx) {
        has_wall = a.wall.flags[(int64_t)yo * a.wall.nchunk + (x >> 5)] != 0;
        if (has_wall) {
          const int64_t n = (int64_t)yo * a.nx + x;
          phie = a.wall.phie[n];
          Sx = a.wall.sx[n];
          Sy = a.wall.sy[n];
          if (a.wall.uwx) {
            uwx = a.wall.uwx[n];
            uwy = a.wall.uwy[n];
          }
        }
      }
      T Fx, Fy;
      node_force<T>(a.phys, rho, ux, uy, psi_c, sfx, sfy, has_wall, phie, Sx, Sy, uwx, uwy,
                    inv_rho, Fx, Fy);

      if (x < a.nx) {
        if (!(fabs(rho) <= T(3.0e38))) atomicOr(a.status, kStatusNonFinite);
        if constexpr (MODE == kModeStep) {
          const T usx = ux + div_rho<T>(Fx, rho, inv_rho);
          const T usy = uy + div_rho<T>(Fy, rho, inv_rho);
          if (a.phys.project) project<Q, T>(f, rho, jx, jy);
          node_collide<Q, T>(a.phys, f, rho, ux, uy, usx, usy);
          // Primary store plus periodic images inside the ghost frame.
          S* out = a.fout;
          const int64_t row = (int64_t)(yo + GY) * a.pitch;
#pragma unroll
          for (int i = 0; i < Q; ++i)
            out[i * a.plane + row + x + GX] = C::enc(f[i], T(L::w(i)) * rho_s);
          const bool edge = x < GX || x >= a.nx - GX || yo < GY || yo >= a.ny - GY;
          if (edge) {
            int xa = x;
            while (xa - a.nx >= -GX) xa -= a.nx;
            int ya = yo;
            while (ya - a.ny >= -GY) ya -= a.ny;
            for (int ym = ya; ym < a.ny + GY; ym += a.ny) {
              for (int xm = xa; xm < a.nx + GX; xm += a.nx) {
                if (xm == x && ym == yo) continue;
                const int64_t off = (int64_t)(ym + GY) * a.pitch + xm + GX;
#pragma unroll
                for (int i = 0; i < Q; ++i)
                  out[i * a.plane + off] = C::enc(f[i], T(L::w(i)) * rho_s);
              }
            }
          }
        } else {
          const int64_t n = (int64_t)yo * a.nx + x;
          const double px = (double)jx + 0.5 * (double)Fx;
          const double py = (double)jy + 0.5 * (double)Fy;
          a.out_rho[n] = (double)rho;
          if (a.momentum) {
            a.out_ux[n] = px;
            a.out_uy[n] = py;
          } else {
            a.out_ux[n] = px / (double)rho;
            a.out_uy[n] = py / (double)rho;
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && k >= R) {
      const int kk = k - R + NS;
      if (kk < K) {
        issue(kk);
        issued = kk + 1;
      }
    }
  }

  if (*s_abort) {
    // A stage never completed.  Record it, then give the copies still in
    // flight a bounded chance to land before the CTA's shared memory goes away.
    if (tid == 0) {
      atomicOr(a.status, kStatusTimeout);
      for (int r = k; r < issued; ++r) mbar_wait_bounded(&bars[r % NS], (uint32_t)(r / NS) & 1u);
    }
  }
}

}  // namespace lbm
