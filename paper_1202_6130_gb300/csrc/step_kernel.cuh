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
// Schedule.  A CTA owns a strip of W columns and a segment of L rows (one
// thread per column, or per pair of columns with packed FP32 arithmetic) and
// marches through the segment one node row at a time, downwards for even
// segments and upwards for odd ones, so that vertically adjacent segments pull
// the rows they share at about the same time (the second pull hits in L2).
// Each row's Q source rows (one per population, shifted by -c_y) and the row's
// wall flags arrive by TMA in one of NS shared-memory stages, several rows
// ahead of use.  psi is computed once per node (plus R halo nodes on each side
// of the strip, by the first 2R threads) into a ring of 2R+2 rows; the
// collision of row k - R then reads its neighbours' psi from the ring.  The
// extra ring row lets one barrier per row order both the ring and the stage
// reuse.  psi never touches HBM; the redundant work is the 2R halo columns and
// rows of each strip segment.
#pragma once

#include <cuda.h>

#include "f2.cuh"
#include "lattice.cuh"
#include "node.cuh"
#include "tma.cuh"

namespace lbm {

enum : uint32_t { kStatusNonFinite = 1u, kStatusTimeout = 2u };

enum StepMode : int {
  kModeStep = 0,      // write post-collision populations to fout
  kModeMoments = 1,   // write rho and u = (j + F/2) / rho (FP64) instead
};

// Which run-time switches of the update are fixed at compile time:
// kFlRuntime reads psi_kind, project and the rounding mode from the
// arguments; kFlExpPlain is the exponential pseudo-potential without the
// projection step, with stochastic rounding for 16-bit storage (the other
// settings run the kFlRuntime kernel).  Both give the same bits.
enum StepFlags : int { kFlRuntime = 0, kFlExpPlain = 1 };

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
  uint64_t wait_ns;    // bound of every stage wait
  uint32_t extra_tx;   // test hook: bytes each stage expects beyond its copies (0 normally)
  // Step counter of the stochastic rounding: two words indexed by the source
  // buffer; a step reads rng[rng_idx] and one CTA writes rng[rng_idx ^ 1] =
  // rng[rng_idx] + 1 for the next step (kModeStep only).
  uint32_t* rng;
  int32_t rng_idx;
  int32_t stochastic;  // 16-bit storage: 1 = stochastic rounding, 0 = nearest-even
};

// Counter of the step about to run (0 unless it is needed).
template <typename S, int MODE, int FL, typename Args>
__device__ __forceinline__ uint32_t step_key(const Args& a) {
  if constexpr (MODE == kModeStep && Codec<S>::kShifted) {
    if (FL == kFlExpPlain || a.stochastic) return a.rng[a.rng_idx];
  }
  return 0u;
}

// Advances the counter for the next step; called by one thread of one CTA.
template <int MODE, typename Args> __device__ __forceinline__ void advance_key(const Args& a) {
  if constexpr (MODE == kModeStep) a.rng[a.rng_idx ^ 1] = a.rng[a.rng_idx] + 1u;
}

// TMA maps of one population buffer, one per distinct box depth of the
// lattice's plane groups (D2Q9 uses one, D2Q21 three).
constexpr int kMaxMaps = 3;
struct PopMaps {
  CUtensorMap m[kMaxMaps];
};

template <int Q, typename S, int W, int NS> struct StepShape {
  using L = Lattice<Q>;
  using P = Planes<Q>;
  using T = typename Codec<S>::T;
  static constexpr int R = L::R;
  static constexpr int GX = ghost_x<S, R>();
  static constexpr int GY = ghost_y<R>();
  static constexpr int BW = W + 2 * GX;  // box width (elements)
  // Planes are grouped by c_y (one group per c_y = -R..R, consecutive planes);
  // each group arrives as one TMA box as deep as the group: D2Q9 groups have
  // 3 planes, D2Q21 groups 1, 3, 3, 7, 3, 3 and 1.  A tensor map fixes its
  // box, so there is one map per distinct depth.  Every box lands in a
  // 128-byte aligned slot of the stage.
  static constexpr int NBOX = 2 * R + 1;
  static constexpr int CHUNKS = W / 32;  // wall-flag words per row
  // The flag words of a strip row arrive as one TMA box of FLAG_BOX words
  // that starts at a multiple of 4 words (16 bytes) at or below the strip's
  // first word; FLAG_BOX covers the strip from any such start.
  static constexpr int flag_box() {
    int need = CHUNKS;
    for (int j = 0; j < 4; ++j) need = (CHUNKS * j) % 4 + CHUNKS > need ? (CHUNKS * j) % 4 + CHUNKS : need;
    return (need + 3) / 4 * 4;
  }
  static constexpr int FLAG_BOX = flag_box();
  static constexpr int FLAG_SLOT = ((FLAG_BOX * 4 + 127) / 128) * 128;
  // Nodes per thread: with FP32 arithmetic (D2Q9; D2Q21 with 16-bit
  // storage) adjacent columns are updated in packed FP32 pairs, one pair per
  // thread; otherwise one node.  (The paired march takes any number of pairs
  // per thread; two pairs, i.e. 32-thread CTAs for 16-bit D2Q9, measured 25%
  // slower than one on GB300.)
  static constexpr int V = (sizeof(T) == 4 && (Q == 9 || sizeof(S) == 2)) ? 2 : 1;
  static constexpr int NT = W / V;                       // threads per CTA
  // Ring column of node 0: at least R, and even for pairs.
  static constexpr int RO = V >= 2 ? (R + 1) / 2 * 2 : R;
  static constexpr int RING_W = W + 2 * RO;
  static constexpr int RING_H = 2 * R + 2;
  static constexpr uint32_t TX_POP = Q * BW * (uint32_t)sizeof(S);
  static constexpr uint32_t TX_FLAGS = FLAG_BOX * 4;
  // Populations of the node row being collided stay in registers (R = 1) or
  // are re-read from its stage (R > 1, where R rows of Q values would not fit).
  static constexpr bool kRegs = (R == 1);
  // Compile-time stage layout: per group j its c_y, first plane, depth, byte
  // offset in the stage and tensor map (by depth); per population i the
  // element offset of its pulled row inside a stage.
  struct Tables {
    int pop_row[Q];
    int box_cy[NBOX];
    int box_plane[NBOX];
    int box_depth[NBOX];
    int box_off[NBOX];
    int box_map[NBOX];
    int depth[kMaxMaps];
    int nmap;
    int pop_bytes;
  };
  static constexpr Tables make_tables() {
    Tables t{};
    int off = 0;
    for (int j = 0; j < NBOX; ++j) {
      const int cy = j - R;
      int first = Q, n = 0;
      for (int i = 0; i < Q; ++i) {
        if (L::cy(i) != cy) continue;
        ++n;
        if (P::kTable.plane[i] < first) first = P::kTable.plane[i];
      }
      t.box_cy[j] = cy;
      t.box_plane[j] = first;
      t.box_depth[j] = n;
      t.box_off[j] = off;
      int k = 0;
      while (k < t.nmap && t.depth[k] != n) ++k;
      if (k == t.nmap) t.depth[t.nmap++] = n;
      t.box_map[j] = k;
      off += (n * BW * (int)sizeof(S) + 127) / 128 * 128;
    }
    t.pop_bytes = off;
    for (int i = 0; i < Q; ++i) {
      const int j = L::cy(i) + R;
      t.pop_row[i] = t.box_off[j] / (int)sizeof(S) + (P::kTable.plane[i] - t.box_plane[j]) * BW;
    }
    return t;
  }
  static constexpr Tables kTab = make_tables();
  static constexpr int NMAP = kTab.nmap;
  static constexpr int POP_BYTES = kTab.pop_bytes;  // flags slot follows the boxes
  static constexpr int STAGE = POP_BYTES + FLAG_SLOT;
  static constexpr int SMEM = 128 /*alignment slack*/ + NS * STAGE + NS * 8 +
                              RING_H * RING_W * (int)sizeof(T) + 16;
  static_assert(W % 32 == 0 && W >= 64 && FLAG_BOX <= 256, "strip width");
  static_assert(NT % 32 == 0 && NT >= 32, "threads per CTA");
  static_assert(NS >= R + 2, "pipeline depth");
  static_assert(NMAP <= kMaxMaps && BW <= 256, "tensor-map boxes");
};

// Shared-memory carve-up of one CTA: NS stages, their mbarriers, the psi ring
// and an abort flag.
template <int Q, typename S, int W, int NS> struct StepSmem {
  using Sh = StepShape<Q, S, W, NS>;
  using T = typename Codec<S>::T;
  unsigned char* stages;
  uint64_t* bars;
  T* ring;
  int* s_abort;
  __device__ static StepSmem carve(unsigned char* raw) {
    StepSmem v;
    // Aligned by an offset from `raw` (not through an integer cast), so that
    // the compiler still sees shared-memory pointers and emits shared loads
    // and stores with 32-bit addresses rather than generic ones.
    unsigned char* base = raw + ((128u - (smem_addr(raw) & 127u)) & 127u);
    v.stages = base;
    v.bars = reinterpret_cast<uint64_t*>(base + NS * Sh::STAGE);
    v.ring = reinterpret_cast<T*>(v.bars + NS);
    v.s_abort = reinterpret_cast<int*>(v.ring + Sh::RING_H * Sh::RING_W);
    return v;
  }
};

// Roles: the first lane of the last warp issues the TMA copies; the first 2R
// threads (all in warp 0) form the psi of the R halo columns on either side.
template <int NT> constexpr int kIssuer = NT - 32;

// Initialises the stage barriers (once per CTA) and returns the L2 policy the
// issuer attaches to its loads.
template <int Q, typename S, int W, int NS>
__device__ __forceinline__ uint64_t step_smem_init(const StepSmem<Q, S, W, NS>& sm) {
  uint64_t policy = 0;
  if (threadIdx.x == kIssuer<StepShape<Q, S, W, NS>::NT>) {
#pragma unroll 1
    for (int s = 0; s < NS; ++s) mbar_init(&sm.bars[s], 1);
    *sm.s_abort = 0;
    fence_barrier_init();
    policy = l2_policy_evict_first();
  }
  __syncthreads();
  return policy;
}

// Advances one strip segment of one lattice by a time step: node rows
// [y0, y0 + Lr) of the W columns starting at x0.  `g` counts the rows this CTA
// has pulled so far (stage g % NS, mbarrier phase (g / NS) & 1) and is
// advanced by Lr + 2R, so a CTA may march several segments in turn.  With
// `rev` the segment is marched upwards (row y0 + Lr + R - 1 first); the node
// arithmetic is the same in either direction.  Returns false if a stage never
// arrived (the status word then has kStatusTimeout).
template <int Q, typename S, int W, int NS, int MODE, int FL, typename Args>
__device__ __forceinline__ bool march_segment(const PopMaps* src, const CUtensorMap* flg,
                                              const Args& a, int x0, int y0, int Lr, bool rev,
                                              const StepSmem<Q, S, W, NS>& sm, uint32_t& g,
                                              uint64_t policy) {
  using Sh = StepShape<Q, S, W, NS>;
  using L = Lattice<Q>;
  using T = typename Codec<S>::T;
  using C = Codec<S>;
  static_assert(!C::kShifted, "16-bit storage runs the paired march");
  constexpr int kPsiKind = FL == kFlExpPlain ? 0 : -1;
  constexpr int R = Sh::R;
  constexpr int GX = Sh::GX;
  constexpr int GY = Sh::GY;
  unsigned char* const stages = sm.stages;
  uint64_t* const bars = sm.bars;
  T* const ring = sm.ring;
  int* const s_abort = sm.s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int K = Lr + 2 * R;  // node rows y0 - R .. y0 + Lr + R - 1
  // Node row of march position k, and the march position offset of the row
  // one above (c_y = +1): +1 marching down, -1 marching up.
  const int ybase = rev ? y0 + Lr + R - 1 : y0 - R;
  const int ds = rev ? -1 : 1;
  const int x = x0 + tid;
  const uint32_t g0 = g;
  const bool wall_on = a.wall.active != 0;
  const bool strip_edge = x0 < GX || x0 + W > a.nx - GX;
  // Every node has at most one periodic image column and one image row.
  const bool simple_images = a.nx >= 2 * GX && a.ny >= 2 * GY;
  const uint32_t tx_bytes = Sh::TX_POP + (wall_on ? Sh::TX_FLAGS : 0u) + a.extra_tx;
  constexpr int kIss = kIssuer<Sh::NT>;

  // Every thread is done with the stages and ring of the previous segment.
  __syncthreads();

  // The issuer copies node row k into stage (g0 + k) % NS: one box per plane
  // group (the group's source row is y - c_y) plus, with walls, the row's flags.
  auto issue = [&](int k) {
    const uint32_t gk = g0 + (uint32_t)k;
    const int s = (int)(gk % NS);
    const int ynode = ybase + ds * k;
    mbar_arrive_expect_tx(&bars[s], tx_bytes);
    unsigned char* st = stages + s * Sh::STAGE;
    static_for<0, Sh::NBOX>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      constexpr int cy = Sh::kTab.box_cy[j];
      // Normal L2 priority: the 2R halo rows of a segment are read again by
      // the segment below a few microseconds later and should hit in L2.
      constexpr int off = Sh::kTab.box_off[j], map = Sh::kTab.box_map[j];
      constexpr int plane = Sh::kTab.box_plane[j];
      tma_load_3d(st + off, &src->m[map], &bars[s], x0, ynode - cy + GY, plane);
    });
    if (wall_on) tma_load_2d(st + Sh::POP_BYTES, flg, &bars[s], (x0 >> 5) & ~3, ynode);
  };
  int issued = 0;
  if (tid == kIss) {
    static_for<0, Sh::NMAP>([&](auto kc) { prefetch_tensormap(&src->m[decltype(kc)::value]); });
    if (wall_on) prefetch_tensormap(flg);
    const int n0 = min(NS, K);
#pragma unroll 1
    for (int k = 0; k < n0; ++k) issue(k);
    issued = n0;
  }
  const int flag0 = (x0 >> 5) & 3;  // the strip's first word in the flag box

  // Population I of node column xl (relative to x0) from a stage: pulled from
  // column xl - c_x of its box row, whose first element is node column -GX.
  auto load_pop = [&](const S* st, auto ic, int xl) -> T {
    constexpr int i = decltype(ic)::value;
    constexpr int off = Sh::kTab.pop_row[i] + GX - L::cx(i);
    return C::load(st[off + xl]);
  };
  auto psi_at = [&](const S* st, int xl) -> T {
    T rho = 0;
    static_for<0, Q>([&](auto ic) {
      const T v = load_pop(st, ic, xl);
      rho = (decltype(ic)::value == 0) ? v : rho + v;
    });
    return pseudo_potential<Q, T, kPsiKind>(a.phys, rho);
  };
  auto flags_of = [&](const unsigned char* st) -> uint32_t {
    return wall_on ? reinterpret_cast<const uint32_t*>(st + Sh::POP_BYTES)[flag0 + warp] : 0u;
  };

  T fnext[Q];            // kRegs: populations of the row whose psi was just formed
  uint32_t flag_next = 0;
  // Stage and mbarrier phase of row k, advanced incrementally.
  int s = (int)(g0 % NS);
  uint32_t phase = (g0 / NS) & 1u;
  int k = 0;
  // With kRegs, unrolled by two so that the populations carried from one row
  // to the next alternate between register sets instead of being copied;
  // otherwise not unrolled (the D2Q21 body is large enough to miss in the
  // instruction cache when duplicated).
  constexpr int kUnroll = Sh::kRegs ? 2 : 1;
#pragma unroll kUnroll
  for (; k < K; ++k) {
    if (!mbar_wait_bounded(&bars[s], phase, a.wait_ns)) *s_abort = 1;
    const unsigned char* stb = stages + s * Sh::STAGE;
    const S* st = reinterpret_cast<const S*>(stb);
    // Populations of the row collided in this iteration (row k - R).
    T f[Q];
    uint32_t flag;
    if constexpr (Sh::kRegs) {
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = fnext[i];
      flag = flag_next;
    }

    // psi of node row k: own column and the halo columns.
    T* ring_row = ring + (k % Sh::RING_H) * Sh::RING_W;
    {
      T rho = 0;
      static_for<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const T v = load_pop(st, ic, tid);
        if constexpr (Sh::kRegs) fnext[i] = v;
        rho = (i == 0) ? v : rho + v;
      });
      ring_row[tid + Sh::RO] = pseudo_potential<Q, T, kPsiKind>(a.phys, rho);
      if constexpr (Sh::kRegs) flag_next = flags_of(stb);
    }
    // The 2R halo columns by the first 2R threads (one warp diverges, not two).
    if (tid < 2 * R) {
      const int xl = tid < R ? tid - R : W + tid - R;
      ring_row[xl + Sh::RO] = psi_at(st, xl);
    }
    __syncthreads();
    if (*s_abort) break;

    // Every thread has finished iteration k - 1: recycle the stage it last used.
    if (tid == kIss) {
      const int fr = k - 1 - (Sh::kRegs ? 0 : R);
      if (fr >= 0 && fr + NS < K) {
        issue(fr + NS);
        issued = fr + NS + 1;
      }
    }

    if (k >= 2 * R) {
      const int ko = k - R;
      const int yo = ybase + ds * ko;
      if constexpr (!Sh::kRegs) {
        const int so = s >= R ? s - R : s - R + NS;  // stage of row k - R
        const unsigned char* sto = stages + so * Sh::STAGE;
        static_for<0, Q>([&](auto ic) {
          f[decltype(ic)::value] = load_pop(reinterpret_cast<const S*>(sto), ic, tid);
        });
        flag = flags_of(sto);
      }
      T rho, jx, jy;
      node_moments<Q, T>(f, rho, jx, jy);
      const T inv_rho = rcp_node<S, T>(rho);
      const T ux = div_rho<T>(jx, rho, inv_rho);
      const T uy = div_rho<T>(jy, rho, inv_rho);

      // sum_i w_i psi(x + c_i) c_i from the ring (rest state contributes 0).
      // prow[R + c_y]: the ring row of node row yo + c_y, at this thread's column.
      static_assert((Sh::RING_H & (Sh::RING_H - 1)) == 0, "ring height is a power of two");
      const T* prow[2 * R + 1];
      static_for<0, 2 * R + 1>([&](auto rc) {
        constexpr int cy = decltype(rc)::value - R;
        prow[R + cy] = ring + ((ko + ds * cy) & (Sh::RING_H - 1)) * Sh::RING_W + tid + Sh::RO;
      });
      const T psi_c = prow[R][0];
      T sfx = 0, sfy = 0;
      static_for<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        if constexpr (L::cx(i) != 0 || L::cy(i) != 0) {
          const T nb = prow[R + L::cy(i)][L::cx(i)];
          const T wn = T(L::w(i)) * nb;
          if constexpr (L::cx(i) != 0) sfx += cmul<L::cx(i)>(wn);
          if constexpr (L::cy(i) != 0) sfy += cmul<L::cy(i)>(wn);
        }
      });

      // Wall terms only on flagged (row, 32-column chunk) pairs.
      const bool has_wall = flag != 0u && x < a.nx;
      T phie = 0, Sx = 0, Sy = 0, uwx = 0, uwy = 0;
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
      T Fx, Fy;
      node_force<T>(a.phys, rho, ux, uy, psi_c, sfx, sfy, has_wall, phie, Sx, Sy, uwx, uwy,
                    inv_rho, Fx, Fy);

      if (x < a.nx) {
        if (!(fabs(rho) <= T(3.0e38))) atomicOr(a.status, kStatusNonFinite);
        if constexpr (MODE == kModeStep) {
          const T usx = ux + div_rho<T>(Fx, rho, inv_rho);
          const T usy = uy + div_rho<T>(Fy, rho, inv_rho);
          if (FL != kFlExpPlain && a.phys.project) project<Q, T>(f, rho, jx, jy);
          node_collide<Q, T>(a.phys, f, rho, ux, uy, usx, usy);
          // The primary store plus periodic images inside the ghost frame.
          S e[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) e[i] = C::store_rn(f[i]);
          S* out = a.fout + (int64_t)(yo + GY) * a.pitch + x + GX;
          static_for<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            out[Planes<Q>::template plane<i> * a.plane] = e[i];
          });
          // Periodic images exist only for nodes within GX of a side or GY of
          // the top or bottom; the strip test is per CTA, the row test per row.
          const bool xedge = strip_edge && (x < GX || x >= a.nx - GX);
          const bool yedge = yo < GY || yo >= a.ny - GY;
          if ((xedge || yedge) && simple_images) {
            // at most one image column (+-nx) and one image row (+-ny)
            const int sx = !xedge ? 0 : (x < GX ? a.nx : -a.nx);
            const int64_t sy = !yedge ? 0 : (int64_t)(yo < GY ? a.ny : -a.ny) * a.pitch;
            auto put = [&](int64_t d) {
              static_for<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                out[d + Planes<Q>::template plane<i> * a.plane] = e[i];
              });
            };
            if (sx != 0) put(sx);
            if (sy != 0) {
              put(sy);
              if (sx != 0) put(sy + sx);
            }
          } else if (xedge || yedge) {
            int xa = x;
            while (xa - a.nx >= -GX) xa -= a.nx;
            int ya = yo;
            while (ya - a.ny >= -GY) ya -= a.ny;
            for (int ym = ya; ym < a.ny + GY; ym += a.ny) {
              for (int xm = xa; xm < a.nx + GX; xm += a.nx) {
                if (xm == x && ym == yo) continue;
                S* o2 = a.fout + (int64_t)(ym + GY) * a.pitch + xm + GX;
                static_for<0, Q>([&](auto ic) {
                  constexpr int i = decltype(ic)::value;
                  o2[Planes<Q>::template plane<i> * a.plane] = e[i];
                });
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
    if (++s == NS) {
      s = 0;
      phase ^= 1u;
    }
  }

  g = g0 + (uint32_t)K;
  if (*s_abort) {
    // A stage never completed.  Record it, then wait (bounded) for the
    // copies still in flight before the shared memory is reused.  Bytes a
    // stage was told to expect beyond its copies (the test hook) are retired
    // first, so each wait ends exactly when its real copies have landed.
    if (tid == kIss) {
      atomicOr(a.status, kStatusTimeout);
      for (int r = k; r < issued; ++r) {
        const uint32_t gr = g0 + (uint32_t)r;
        if (a.extra_tx) mbar_complete_tx(&bars[gr % NS], a.extra_tx);
        mbar_wait_bounded(&bars[gr % NS], (gr / NS) & 1u, a.wait_ns);
      }
    }
    return false;
  }
  return true;
}

// Two nodes per thread (FP32 arithmetic): thread t updates columns 2t and
// 2t + 1 of the strip.  Same schedule and stage layout as march_segment; the
// node arithmetic runs on packed FP32 pairs, aligned pairs of stored
// populations and of psi are moved with one 64- or 32-bit access, and each
// population row is stored as pairs.  With R = 1 (D2Q9) the populations of a
// row stay in registers from its psi pass to its collision; with R > 1
// (D2Q21) the collision re-reads them from the row's stage, as march_segment
// does.  Wall terms, ghost images, the halo psi and a pair that straddles the
// lattice's right edge fall back to per-node code.
template <int Q, typename S, int W, int NS, int MODE, int FL, typename Args>
__device__ __forceinline__ bool march_segment_v2(const PopMaps* src, const CUtensorMap* flg,
                                                 const Args& a, int x0, int y0, int Lr, bool rev,
                                                 const StepSmem<Q, S, W, NS>& sm, uint32_t& g) {
  using Sh = StepShape<Q, S, W, NS>;
  using L = Lattice<Q>;
  using E = EqConst<Q>;
  using C = Codec<S>;
  using PR = Pair<S>;
  using T = float;
  constexpr int R = Sh::R;
  constexpr int GX = Sh::GX;
  constexpr int GY = Sh::GY;
  constexpr int RO = Sh::RO;
  constexpr int P = Sh::V / 2;  // node pairs per thread
  constexpr bool kRegs = Sh::kRegs;
  static_assert(Sh::V % 2 == 0 && RO % 2 == 0 && RO >= R, "paired march");
  constexpr int kPsiKind = FL == kFlExpPlain ? 0 : -1;
  constexpr bool kFastExp = C::kShifted;
  unsigned char* const stages = sm.stages;
  uint64_t* const bars = sm.bars;
  T* const ring = sm.ring;
  int* const s_abort = sm.s_abort;

  const int tid = threadIdx.x;
  const int xa = Sh::V * tid;  // first of the thread's columns, relative to x0
  const int x = x0 + xa;
  const int K = Lr + 2 * R;
  const int ybase = rev ? y0 + Lr + R - 1 : y0 - R;
  const int ds = rev ? -1 : 1;
  const uint32_t g0 = g;
  const bool wall_on = a.wall.active != 0;
  const bool strip_edge = x0 < GX || x0 + W > a.nx - GX;
  // Every node has at most one periodic image column and one image row, and
  // the images of a node pair are a pair again (even nx): the paired store of
  // the ghost images applies.
  const bool simple_images = a.nx >= 2 * GX && a.ny >= 2 * GY && (a.nx & 1) == 0;
  const uint32_t tx_bytes = Sh::TX_POP + (wall_on ? Sh::TX_FLAGS : 0u) + a.extra_tx;
  constexpr int kIss = kIssuer<Sh::NT>;
  const uint32_t key = step_key<S, MODE, FL>(a);

  __syncthreads();

  auto issue = [&](int k) {
    const uint32_t gk = g0 + (uint32_t)k;
    const int s = (int)(gk % NS);
    const int ynode = ybase + ds * k;
    mbar_arrive_expect_tx(&bars[s], tx_bytes);
    unsigned char* st = stages + s * Sh::STAGE;
    static_for<0, Sh::NBOX>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      constexpr int cy = Sh::kTab.box_cy[j];
      constexpr int off = Sh::kTab.box_off[j], map = Sh::kTab.box_map[j];
      constexpr int plane = Sh::kTab.box_plane[j];
      tma_load_3d(st + off, &src->m[map], &bars[s], x0, ynode - cy + GY, plane);
    });
    if (wall_on) tma_load_2d(st + Sh::POP_BYTES, flg, &bars[s], (x0 >> 5) & ~3, ynode);
  };
  int issued = 0;
  if (tid == kIss) {
    static_for<0, Sh::NMAP>([&](auto kc) { prefetch_tensormap(&src->m[decltype(kc)::value]); });
    if (wall_on) prefetch_tensormap(flg);
    const int n0 = min(NS, K);
#pragma unroll 1
    for (int k = 0; k < n0; ++k) issue(k);
    issued = n0;
  }
  const int flag0 = (x0 >> 5) & 3;  // the strip's first word in the flag box

  // Stored value I of the columns of pair p (f, or the scaled deviation h for
  // 16-bit storage): an aligned pair when c_x is even (one access), else two
  // single loads.
  auto load_pair = [&](const S* st, auto ic, int p) -> F2 {
    constexpr int i = decltype(ic)::value;
    constexpr int off = Sh::kTab.pop_row[i] + GX - L::cx(i);
    const int xc = xa + 2 * p;
    if constexpr ((off & 1) == 0) {
      return PR::load(*reinterpret_cast<const typename PR::Raw*>(st + off + xc));
    } else {
      return PR::load1(st[off + xc], st[off + xc + 1]);
    }
  };
  // rho from the sum H of a node's stored values: H itself, or for 16-bit
  // storage H / sigma + rho_s (the shifts w_i rho_s sum to rho_s).
  constexpr T kInvScale = T(1) / T(C::kScale);
  auto rho_of = [&](T H) -> T {
    if constexpr (C::kShifted) return fmaf(H, kInvScale, a.phys.rho_s);
    else return H;
  };
  auto rho_of2 = [&](F2 H) -> F2 {
    if constexpr (C::kShifted) return fma2(H, F2::splat(kInvScale), F2::splat(a.phys.rho_s));
    else return H;
  };
  auto psi_at = [&](const S* st, int xl) -> T {  // one node (halo columns)
    T H = 0;
    static_for<0, Q>([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      constexpr int off = Sh::kTab.pop_row[i] + GX - L::cx(i);
      const T v = C::load(st[off + xl]);
      H = (i == 0) ? v : H + v;
    });
    return pseudo_potential<Q, T, kPsiKind, kFastExp>(a.phys, rho_of(H));
  };

  // The thread's columns lie in one 32-column flag chunk.
  auto flags_of = [&](const unsigned char* stage) -> uint32_t {
    return wall_on ? reinterpret_cast<const uint32_t*>(stage + Sh::POP_BYTES)[flag0 + (xa >> 5)]
                   : 0u;
  };

  // kRegs: stored values and their sum H (formed once, in table order) of the
  // row whose psi was just formed, collided in the next iteration.
  F2 fnext[kRegs ? P : 1][kRegs ? Q : 1];
  F2 rho_next[P];
  uint32_t flag_next = 0;
  int s = (int)(g0 % NS);
  uint32_t phase = (g0 / NS) & 1u;
  int k = 0;
  // With kRegs, unrolled by two so that the carried registers alternate
  // between two sets instead of being copied.
  constexpr int kUnroll = kRegs ? 2 : 1;
#pragma unroll kUnroll
  for (; k < K; ++k) {
    if (!mbar_wait_bounded(&bars[s], phase, a.wait_ns)) *s_abort = 1;
    const unsigned char* stb = stages + s * Sh::STAGE;
    const S* st = reinterpret_cast<const S*>(stb);

    // Populations, rho and wall flags of the row collided in this iteration
    // (row k - R).
    F2 f[P][Q];
    F2 rho_cur[P];
    uint32_t flag = 0;
    if constexpr (kRegs) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[p][i] = fnext[p][i];
        rho_cur[p] = rho_next[p];
      }
      flag = flag_next;
    }

    // psi of node row k for the thread's columns, then the halo columns.
    T* ring_row = ring + (k % Sh::RING_H) * Sh::RING_W;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      F2 H;
      static_for<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const F2 v = load_pair(st, ic, p);
        if constexpr (kRegs) fnext[p][i] = v;
        H = (i == 0) ? v : H + v;
      });
      const F2 rho = rho_of2(H);
      float2 psi2;
      if constexpr (kPsiKind == 0 && kFastExp) {
        // psi_exp_fast of both nodes, the product and the fused
        // multiply-add packed
        const F2 e2 = rho * F2::splat(a.phys.exp2_scale);
        psi2 = fma2(F2(ex2_approx(e2.x()), ex2_approx(e2.y())), F2::splat(-a.phys.rho0),
                    F2::splat(a.phys.rho0)).v;
      } else {
        psi2 = make_float2(pseudo_potential<Q, T, kPsiKind, kFastExp>(a.phys, rho.x()),
                           pseudo_potential<Q, T, kPsiKind, kFastExp>(a.phys, rho.y()));
      }
      *reinterpret_cast<float2*>(ring_row + RO + xa + 2 * p) = psi2;
      if constexpr (kRegs) rho_next[p] = H;
    }
    if constexpr (kRegs) flag_next = flags_of(stb);
    if (tid < 2 * R) {
      const int xl = tid < R ? tid - R : W + tid - R;
      ring_row[xl + RO] = psi_at(st, xl);
    }
    __syncthreads();
    if (*s_abort) break;

    // Every thread has finished iteration k - 1: recycle the stage it last used.
    if (tid == kIss) {
      const int fr = k - 1 - (kRegs ? 0 : R);
      if (fr >= 0 && fr + NS < K) {
        issue(fr + NS);
        issued = fr + NS + 1;
      }
    }

    if (k >= 2 * R) {
      const int ko = k - R;
      const int yo = ybase + ds * ko;
      if constexpr (!kRegs) {
        const int so = s >= R ? s - R : s - R + NS;  // stage of row k - R
        const unsigned char* sto = stages + so * Sh::STAGE;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          static_for<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            f[p][i] = load_pair(reinterpret_cast<const S*>(sto), ic, p);
            rho_cur[p] = (i == 0) ? f[p][i] : rho_cur[p] + f[p][i];
          });
        }
        flag = flags_of(sto);
      }
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int xp = x + 2 * p;           // first column of pair p
        const bool pair_ok = xp + 1 < a.nx;  // both nodes exist
        // f_: the stored values (f, or h = sigma (f - w rho_s) for 16-bit
        // storage).  H: their sum in table order (the psi pass's sum), rho
        // from it; J = sum f_i c_i (D2Q9: the diagonal differences f5 - f7
        // and f8 - f6 shared by its two components; otherwise in table
        // order), j = J / sigma (the shifts carry no momentum).
        F2 (&f_)[Q] = f[p];
        const F2 Hm = rho_cur[p];
        const F2 rho = rho_of2(Hm);
        F2 Jx, Jy;
        if constexpr (Q == 9) {
          const F2 d57 = f_[5] - f_[7], d86 = f_[8] - f_[6];
          Jx = ((f_[1] - f_[3]) + d57) + d86;
          Jy = ((f_[2] - f_[4]) + d57) - d86;
        } else {
          Jx = F2::splat(0.f);
          Jy = F2::splat(0.f);
          static_for<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if constexpr (L::cx(i) != 0) Jx = fma2(f_[i], F2::splat(T(L::cx(i))), Jx);
            if constexpr (L::cy(i) != 0) Jy = fma2(f_[i], F2::splat(T(L::cy(i))), Jy);
          });
        }
        F2 jx = Jx, jy = Jy;
        if constexpr (C::kShifted && C::kScale != 1.0f) {
          jx = Jx * F2::splat(kInvScale);
          jy = Jy * F2::splat(kInvScale);
        }
        const F2 inv_rho(rcp_node<S, float>(rho.x()), rcp_node<S, float>(rho.y()));
        const F2 ux = jx * inv_rho;
        const F2 uy = jy * inv_rho;

        // Neighbour psi, sum_i w_i psi(x + c_i) c_i.
        F2 sfx = F2::splat(0.f), sfy = F2::splat(0.f), psi_c;
        if constexpr (Q != 9) {
          // Ring row of node row yo + c_y; the psi pair at column offset c_x
          // is one aligned pair (c_x even) or the halves of two.
          auto ring_at = [&](int cy, int o) -> float2 {
            return *reinterpret_cast<const float2*>(
                ring + ((ko + ds * cy) & (Sh::RING_H - 1)) * Sh::RING_W + RO + xa + 2 * p + o);
          };
          psi_c = F2(ring_at(0, 0));
          static_for<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int cx = L::cx(i), cy = L::cy(i);
            if constexpr (i == L::REST) return;
            F2 nb;
            if constexpr ((cx & 1) == 0) {
              nb = F2(ring_at(cy, cx));
            } else {
              nb = F2(ring_at(cy, cx - 1).y, ring_at(cy, cx + 1).x);
            }
            if constexpr (cx != 0) sfx = fma2(nb, F2::splat(T(L::w(i) * cx)), sfx);
            if constexpr (cy != 0) sfy = fma2(nb, F2::splat(T(L::w(i) * cy)), sfy);
          });
        } else {
          // D2Q9: three aligned pairs per ring row cover the pair's columns
          // and one more on either side.
          static_for<0, 3>([&](auto rc) {
            constexpr int cy = decltype(rc)::value - 1;
            const T* row = ring + ((ko + ds * cy) & (Sh::RING_H - 1)) * Sh::RING_W + RO + xa + 2 * p;
            const float2 A = *reinterpret_cast<const float2*>(row - 2);
            const float2 B = *reinterpret_cast<const float2*>(row);
            const float2 Cc = *reinterpret_cast<const float2*>(row + 2);
            const F2 pm(A.y, B.x), p0(B), pp(B.y, Cc.x);   // psi at c_x = -1, 0, +1
            if constexpr (cy == 0) {
              psi_c = p0;
              sfx = fma2(pp - pm, F2::splat(T(L::w(1))), sfx);  // (1,0) and (-1,0)
            } else {
              // (0,cy): weight w_axis; (+-1, cy): weight w_diag
              constexpr T sg = cy > 0 ? T(1) : T(-1);
              sfy = fma2(p0, F2::splat(sg * T(L::w(2))), sfy);
              sfy = fma2(pp + pm, F2::splat(sg * T(L::w(5))), sfy);
              sfx = fma2(pp - pm, F2::splat(T(L::w(5))), sfx);
            }
          });
        }

        // Force: F_FF, then the wall terms on flagged chunks, then body force.
        const F2 mg = F2::splat(-a.phys.G) * psi_c;
        F2 Fx, Fy;
        if (flag != 0u) {
          const F2 ffx = mg * sfx, ffy = mg * sfy;
          T phe[2] = {0, 0}, Sx[2] = {0, 0}, Sy[2] = {0, 0}, wx[2] = {0, 0}, wy[2] = {0, 0};
  #pragma unroll
          for (int e = 0; e < 2; ++e) {
            if (xp + e < a.nx) {
              const int64_t n = (int64_t)yo * a.nx + xp + e;
              phe[e] = a.wall.phie[n];
              Sx[e] = a.wall.sx[n];
              Sy[e] = a.wall.sy[n];
              if (a.wall.uwx) {
                wx[e] = a.wall.uwx[n];
                wy[e] = a.wall.uwy[n];
              }
            }
          }
          const F2 rp = rho * F2(phe[0], phe[1]);
          const F2 dfx = rp * (F2(wx[0], wx[1]) - ux - ffx * inv_rho);
          const F2 dfy = rp * (F2(wy[0], wy[1]) - uy - ffy * inv_rho);
          Fx = ((ffx + rho * F2(Sx[0], Sx[1])) + dfx) + F2::splat(a.phys.bfx);
          Fy = ((ffy + rho * F2(Sy[0], Sy[1])) + dfy) + F2::splat(a.phys.bfy);
        } else {
          Fx = fma2(mg, sfx, F2::splat(a.phys.bfx));
          Fy = fma2(mg, sfy, F2::splat(a.phys.bfy));
        }

        if (xp < a.nx) {
          if (!(fabsf(rho.x()) <= 3.0e38f) || (pair_ok && !(fabsf(rho.y()) <= 3.0e38f)))
            atomicOr(a.status, kStatusNonFinite);
          if constexpr (MODE == kModeStep) {
            const F2 usx = fma2(Fx, inv_rho, ux);
            const F2 usy = fma2(Fy, inv_rho, uy);
            // EDM-BGK in pair form (see node_collide), packed over the two nodes
            // and written as fused multiply-adds: with ca = c.(u* - g u) / theta
            // and sb = omega - B + ((c.u*)^2 - g (c.u)^2) / (2 theta^2),
            // f_post(+-c) = g f(+-c) + w rho (sb +- ca).
            const F2 gg = F2::splat(a.phys.one_m_omega), ngg = F2::splat(-a.phys.one_m_omega);
            const F2 ax3 = fma2(ngg, ux, usx) * F2::splat(T(E::inv_theta));
            const F2 ay3 = fma2(ngg, uy, usy) * F2::splat(T(E::inv_theta));
            const F2 us2 = fma2(usy, usy, usx * usx), u2 = fma2(uy, uy, ux * ux);
            const F2 wB = fma2(fma2(ngg, u2, us2), F2::splat(-T(E::inv_2theta)),
                               F2::splat(a.phys.omega));
            if (FL != kFlExpPlain && a.phys.project) {
              // rare path: per node.  The projection is linear and maps the
              // shift w_i rho_s to itself, so it acts on h with (H, J) as it
              // acts on f with (rho, j).
              T fa[Q], fb[Q];
  #pragma unroll
              for (int i = 0; i < Q; ++i) {
                fa[i] = f_[i].x();
                fb[i] = f_[i].y();
              }
              project<Q, T>(fa, Hm.x(), Jx.x(), Jy.x());
              project<Q, T>(fb, Hm.y(), Jx.y(), Jy.y());
  #pragma unroll
              for (int i = 0; i < Q; ++i) f_[i] = F2(fa[i], fb[i]);
            }
            if constexpr (C::kShifted) {
              // The same update on h = sigma (f - w rho_s):
              //   h_post(+-c) = g h(+-c) + sigma w [rho (sb +- ca) - omega rho_s].
              const F2 nwr = F2::splat(a.phys.neg_omega_rho_s);
              static_for<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int j = opposite<Q>(i);
                if constexpr (i != L::REST && i < j) {
                  const F2 cs = cdot2<L::cx(i), L::cy(i)>(usx, usy);
                  const F2 cu = cdot2<L::cx(i), L::cy(i)>(ux, uy);
                  const F2 ca = cdot2<L::cx(i), L::cy(i)>(ax3, ay3);
                  const F2 t = fma2(ngg, cu * cu, cs * cs);
                  const F2 sb = fma2(t, F2::splat(T(E::inv_2theta2)), wB);
                  const F2 z = fma2(rho, sb, nwr);
                  const F2 sw = F2::splat(T(C::kScale * L::w(i)));
                  const F2 hi = fma2(gg, f_[i], sw * fma2(rho, ca, z));
                  const F2 hj = fma2(gg, f_[j], sw * fma2(rho, -ca, z));
                  f_[i] = hi;
                  f_[j] = hj;
                }
              });
            } else {
              static_for<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr int j = opposite<Q>(i);
                // The rest population comes from the mass closure below.
                if constexpr (i != L::REST && i < j) {
                  const F2 cs = cdot2<L::cx(i), L::cy(i)>(usx, usy);
                  const F2 cu = cdot2<L::cx(i), L::cy(i)>(ux, uy);
                  const F2 ca = cdot2<L::cx(i), L::cy(i)>(ax3, ay3);
                  const F2 wr = F2::splat(T(L::w(i))) * rho;
                  const F2 t = fma2(ngg, cu * cu, cs * cs);
                  const F2 sb = fma2(t, F2::splat(T(E::inv_2theta2)), wB);
                  const F2 fi = fma2(gg, f_[i], wr * (sb + ca));
                  const F2 fj = fma2(gg, f_[j], wr * (sb - ca));
                  f_[i] = fi;
                  f_[j] = fj;
                }
              });
            }
            {  // mass closure of the rest population: the stored values sum to
               // H (rho, or sigma (rho - rho_s) for 16-bit storage) after the
               // collision as before it
              constexpr int i0 = L::REST == 0 ? 1 : 0;
              F2 moving = f_[i0];
#pragma unroll
              for (int i = i0 + 1; i < Q; ++i)
                if (i != L::REST) moving += f_[i];
              f_[L::REST] = Hm - moving;
            }
            // Round both nodes once (stochastic rounding: bits from the node
            // pair and the step), then the primary store plus periodic images.
            typename PR::Raw raw[Q];
            if constexpr (C::kShifted) {
              if (FL == kFlExpPlain || a.stochastic) {
                const uint32_t h = sr_hash((uint32_t)xp, (uint32_t)yo, key);
                static_for<0, Q>([&](auto ic) {
                  constexpr int i = decltype(ic)::value;
                  raw[i] = PR::store_sr(f_[i], h * sr_multiplier(i));
                });
              } else {
  #pragma unroll
                for (int i = 0; i < Q; ++i) raw[i] = PR::store_rn(f_[i]);
              }
            } else {
  #pragma unroll
              for (int i = 0; i < Q; ++i) raw[i] = PR::store_rn(f_[i]);
            }
            S* out = a.fout + (int64_t)(yo + GY) * a.pitch + xp + GX;
            if (pair_ok) {
              static_for<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                *reinterpret_cast<typename PR::Raw*>(out + Planes<Q>::template plane<i> * a.plane) =
                    raw[i];
              });
            } else {
              static_for<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                out[Planes<Q>::template plane<i> * a.plane] = PR::lane(raw[i], 0);
              });
            }
            const bool xedge = strip_edge && (xp < GX || xp + 1 >= a.nx - GX);
            const bool yedge = yo < GY || yo >= a.ny - GY;
            if ((xedge || yedge) && pair_ok && simple_images) {
              // Both nodes of the pair have the same images: at most one
              // column shift (+-nx) and one row shift (+-ny), stored as pairs.
              const int sx = !xedge ? 0 : (xp < GX ? a.nx : -a.nx);
              const int64_t sy = !yedge ? 0 : (int64_t)(yo < GY ? a.ny : -a.ny) * a.pitch;
              auto put = [&](int64_t d) {
                static_for<0, Q>([&](auto ic) {
                  constexpr int i = decltype(ic)::value;
                  *reinterpret_cast<typename PR::Raw*>(out + d + Planes<Q>::template plane<i> * a.plane) =
                      raw[i];
                });
              };
              if (sx != 0) put(sx);
              if (sy != 0) {
                put(sy);
                if (sx != 0) put(sy + sx);
              }
            } else if (xedge || yedge) {
  #pragma unroll 1
              for (int e = 0; e < 2; ++e) {
                const int xn = xp + e;
                if (xn >= a.nx) break;
                int xs = xn;
                while (xs - a.nx >= -GX) xs -= a.nx;
                int ya = yo;
                while (ya - a.ny >= -GY) ya -= a.ny;
                for (int ym = ya; ym < a.ny + GY; ym += a.ny) {
                  for (int xm = xs; xm < a.nx + GX; xm += a.nx) {
                    if (xm == xn && ym == yo) continue;
                    S* o2 = a.fout + (int64_t)(ym + GY) * a.pitch + xm + GX;
                    static_for<0, Q>([&](auto ic) {
                      constexpr int i = decltype(ic)::value;
                      o2[Planes<Q>::template plane<i> * a.plane] = PR::lane(raw[i], e);
                    });
                  }
                }
              }
            }
          } else {
  #pragma unroll
            for (int e = 0; e < 2; ++e) {
              if (xp + e >= a.nx) break;
              const int64_t n = (int64_t)yo * a.nx + xp + e;
              const double r = e == 0 ? rho.x() : rho.y();
              const double px = (double)(e == 0 ? jx.x() : jx.y()) + 0.5 * (double)(e == 0 ? Fx.x() : Fx.y());
              const double py = (double)(e == 0 ? jy.x() : jy.y()) + 0.5 * (double)(e == 0 ? Fy.x() : Fy.y());
              a.out_rho[n] = r;
              if (a.momentum) {
                a.out_ux[n] = px;
                a.out_uy[n] = py;
              } else {
                a.out_ux[n] = px / r;
                a.out_uy[n] = py / r;
              }
            }
          }
        }
      }  // pairs
    }
    if (++s == NS) {
      s = 0;
      phase ^= 1u;
    }
  }

  g = g0 + (uint32_t)K;
  if (*s_abort) {
    if (tid == kIss) {
      atomicOr(a.status, kStatusTimeout);
      for (int r = k; r < issued; ++r) {
        const uint32_t gr = g0 + (uint32_t)r;
        if (a.extra_tx) mbar_complete_tx(&bars[gr % NS], a.extra_tx);
        mbar_wait_bounded(&bars[gr % NS], (gr / NS) & 1u, a.wait_ns);
      }
    }
    return false;
  }
  return true;
}

// Marches one segment with the variant the shape selects (one or two nodes
// per thread).
template <int Q, typename S, int W, int NS, int MODE, int FL, typename Args>
__device__ __forceinline__ bool march_any(const PopMaps* src, const CUtensorMap* flg,
                                          const Args& a, int x0, int y0, int Lr, bool rev,
                                          const StepSmem<Q, S, W, NS>& sm, uint32_t& g,
                                          uint64_t policy) {
  if constexpr (StepShape<Q, S, W, NS>::V >= 2)
    return march_segment_v2<Q, S, W, NS, MODE, FL>(src, flg, a, x0, y0, Lr, rev, sm, g);
  else
    return march_segment<Q, S, W, NS, MODE, FL>(src, flg, a, x0, y0, Lr, rev, sm, g, policy);
}

// One time step of one lattice: CTA (bx, by) marches strip bx, segment by.
// Odd segments march upwards, so two vertically adjacent segments, which run
// at about the same time, pull the rows they share (the 2R halo rows of their
// common edge) both at their start or both at their end: the second pull of
// such a row is an L2 hit instead of a DRAM read.
template <int Q, typename S, int W, int NS, int MODE, int MINB, int FL>
__global__ void __launch_bounds__(StepShape<Q, S, W, NS>::NT, MINB)
    step_kernel(const __grid_constant__ PopMaps src, const __grid_constant__ CUtensorMap flg,
                const StepArgs<typename Codec<S>::T, S> a) {
  extern __shared__ unsigned char smem_raw[];
  const auto sm = StepSmem<Q, S, W, NS>::carve(smem_raw);
  const uint64_t policy = step_smem_init(sm);
  const int y0 = blockIdx.y * a.tile_rows;
  uint32_t g = 0;
  // Launched as a programmatic dependent of the previous step: the next step's
  // CTAs may be scheduled as this grid's last wave drains; every global read
  // or write (populations, the step counter, the status word) follows the
  // wait for the previous grid.
  griddep_launch_dependents();
  griddep_wait();
  // Every CTA reads the counter in march_any before this launch ends; the
  // word written here is read only by the next step.
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) advance_key<MODE>(a);
  march_any<Q, S, W, NS, MODE, FL>(&src, &flg, a, blockIdx.x * W, y0, min(a.tile_rows, a.ny - y0),
                               (blockIdx.y & 1u) != 0u, sm, g, policy);
}

// A lattice of a batch: TMA maps of its two population buffers and of its wall
// flags (in device memory; map[d] reads buffer d).
template <typename T, typename S> struct BatchMember {
  PopMaps map[2];
  CUtensorMap flags;
};

// Step arguments of up to kChunk members of a batch for either direction
// (a[m][d] reads buffer d and writes buffer 1 - d), the buffer holding each
// member's state at parity 0, and the chunk's tiles: member m owns tiles
// [tile0[m], tile0[m + 1]), nseg[m] segments of nstrip[m] strips numbered
// segment by segment (tile0[m] = the chunk's tile count past its last member).
// Passed as a kernel parameter, so the kernel reads them from constant memory
// with the CTA-uniform member index that it derives from its block index.
// kChunk: 64 members with FP32 arithmetic, 32 with FP64 (the larger FP64
// arguments), so that the block stays below the 32,764-byte parameter limit.
template <typename T> constexpr int batch_chunk() { return sizeof(T) == 8 ? 32 : 64; }
template <typename T, typename S> struct BatchArgs {
  static constexpr int kChunk = batch_chunk<T>();
  StepArgs<T, S> a[kChunk][2];
  int32_t cur[kChunk];
  int32_t tile0[kChunk + 1];
  int32_t nstrip[kChunk];
  int32_t nseg[kChunk];
};
static_assert(sizeof(BatchArgs<float, float>) <= 32764 && sizeof(BatchArgs<double, double>) <= 32764,
              "batch arguments fit the kernel parameter space");

// One time step of up to kChunk lattices of a batch.  Tile t is segment
// t / nstrip (rows balanced over the member's height, odd segments marched
// upwards as in step_kernel) and strip t % nstrip of its member.  With
// PERSIST, CTA b marches tiles b, b + gridDim.x, ...; otherwise CTA b marches
// tile b.  `parity` flips the read/write buffers on alternate steps.  FL as
// for step_kernel (kFlExpPlain when every member of the chunk has those
// settings).
template <int Q, typename S, int W, int NS, int MINB, bool PERSIST, int FL>
__global__ void __launch_bounds__(StepShape<Q, S, W, NS>::NT, MINB)
    batch_step_kernel(const __grid_constant__ BatchArgs<typename Codec<S>::T, S> P,
                      const BatchMember<typename Codec<S>::T, S>* __restrict__ members,
                      int32_t parity) {
  extern __shared__ unsigned char smem_raw[];
  const auto sm = StepSmem<Q, S, W, NS>::carve(smem_raw);
  const uint64_t policy = step_smem_init(sm);
  uint32_t g = 0;
  // A programmatic dependent of the chunk's previous step (see step_kernel).
  griddep_launch_dependents();
  griddep_wait();
  auto march_tile = [&](int t) -> bool {
    int m = 0;
#pragma unroll
    for (int j = 1; j < P.kChunk; ++j) m += t >= P.tile0[j] ? 1 : 0;
    const int local = t - P.tile0[m];
    const int seg = local / P.nstrip[m];
    const int x0 = (local - seg * P.nstrip[m]) * W;
    const int dir = (P.cur[m] ^ parity) & 1;
    const auto& a = P.a[m][dir];
    const int y0 = (int)((int64_t)a.ny * seg / P.nseg[m]);
    const int y1 = (int)((int64_t)a.ny * (seg + 1) / P.nseg[m]);
    if (threadIdx.x == 0 && local == 0) advance_key<kModeStep>(a);
    const auto* mb = &members[m];
    return march_any<Q, S, W, NS, kModeStep, FL>(&mb->map[dir], &mb->flags, a, x0, y0, y1 - y0,
                                                (seg & 1) != 0, sm, g, policy);
  };
  if constexpr (PERSIST) {
    const int nt = P.tile0[P.kChunk];
#pragma unroll 1
    for (int t = blockIdx.x; t < nt; t += gridDim.x)
      if (!march_tile(t)) return;
  } else {
    march_tile((int)blockIdx.x);
  }
}

}  // namespace lbm
