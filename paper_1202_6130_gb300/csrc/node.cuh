// Per-node arithmetic of the wetting model (Sec. II of arXiv:1202.6130):
// storage codecs, pseudo-potentials, second-order equilibrium, projection and
// the exact-difference-method BGK collision.  Shared by the fused step kernel
// and by the read-out kernels, so that moments are computed with exactly the
// arithmetic the step uses.
#pragma once

#include <cmath>
#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lattice.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Storage codecs.  FP64 / FP32 store f directly.  FP16S / BF16S store the
// scaled deviation h_i = sigma (f_i - w_i rho_s) from the shift w_i rho_s in 16
// bits, with sigma = kHalfScale = 2^8 for FP16S (deviations down to 2.4e-7
// stay in the normal range of binary16, and up to 256 fit) and sigma = 1 for
// BF16S.  The step computes on h itself in FP32: rho = sum_i h_i / sigma +
// rho_s (the weights sum to one), j = sum_i h_i c_i / sigma (the shift carries
// no momentum), and the collision and the projection map deviations to
// deviations, so no per-population shift is ever added or subtracted in FP32.
// The conversion to 16 bits rounds to nearest-even or stochastically: random
// bits are added below the kept mantissa of the FP32 value and the sum is
// truncated, so the stored value rounds up with probability equal to the
// discarded fraction and its expectation is the FP32 value (subnormal results
// included; overflow gives inf).  Round-to-nearest loses every per-step
// increment smaller than half a unit in the last place (a body force of 1e-6
// adds about 3e-7 per population); the stochastic version keeps them on
// average.  Set-up and read-out convert between f and h in FP64 (enc_host,
// dec_host), with the shift w_i rho_s formed in FP64 from the same rho_s the
// step uses.
// ---------------------------------------------------------------------------

// Stochastic-rounding conversions of the sm_100 family: two FP32 values to a
// 16-bit pair, `hi` into the upper half.  As measured on GB300, the lower half
// takes its random bits from r[12:0] (binary16) or r[15:0] (bfloat16) and the
// upper half from r[28:16] or r[31:16].
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float hi, float lo, uint32_t r) {
  uint32_t u;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(u) : "f"(hi), "f"(lo), "r"(r));
  return u;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float hi, float lo, uint32_t r) {
  uint32_t u;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(u) : "f"(hi), "f"(lo), "r"(r));
  return u;
}

constexpr float kHalfScale = 256.0f;
constexpr float kHalfInvScale = 1.0f / 256.0f;

// load: the stored value in the compute type (f, or the scaled deviation h);
// store_rn / store_sr: back to storage (h rounded to 16 bits for FP16S and
// BF16S); enc_host / dec_host: FP64 f <-> storage given the shift w_i rho_s.
template <typename S> struct Codec;

template <> struct Codec<double> {
  using T = double;
  static constexpr bool kShifted = false;
  static constexpr double kScale = 1.0;
  __device__ __forceinline__ static T load(double v) { return v; }
  __device__ __forceinline__ static double store_rn(T v) { return v; }
  __device__ __forceinline__ static double store_sr(T v, uint32_t) { return v; }
  __host__ __device__ static double enc_host(double f, double) { return f; }
  __host__ __device__ static double dec_host(double v, double) { return v; }
};

template <> struct Codec<float> {
  using T = float;
  static constexpr bool kShifted = false;
  static constexpr float kScale = 1.0f;
  __device__ __forceinline__ static T load(float v) { return v; }
  __device__ __forceinline__ static float store_rn(T v) { return v; }
  __device__ __forceinline__ static float store_sr(T v, uint32_t) { return v; }
  __host__ __device__ static float enc_host(double f, double) { return (float)f; }
  __host__ __device__ static double dec_host(float v, double) { return (double)v; }
};

template <> struct Codec<__half> {
  using T = float;
  static constexpr bool kShifted = true;
  static constexpr float kScale = kHalfScale;
  __device__ __forceinline__ static T load(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half store_rn(T h) { return __float2half_rn(h); }
  // r: random word (bits 12..0 are used).
  __device__ __forceinline__ static __half store_sr(T h, uint32_t r) {
    return __ushort_as_half((unsigned short)(cvt_rs_f16x2(0.0f, h, r) & 0xFFFFu));
  }
  __device__ static __half enc_host(double f, double shift) {
    return __double2half((f - shift) * (double)kHalfScale);
  }
  __device__ static double dec_host(__half v, double shift) {
    return (double)__half2float(v) * (double)kHalfInvScale + shift;
  }
};

template <> struct Codec<__nv_bfloat16> {
  using T = float;
  static constexpr bool kShifted = true;
  static constexpr float kScale = 1.0f;
  __device__ __forceinline__ static T load(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 store_rn(T h) { return __float2bfloat16_rn(h); }
  // r: random word (bits 15..0 are used).
  __device__ __forceinline__ static __nv_bfloat16 store_sr(T h, uint32_t r) {
    return __ushort_as_bfloat16((unsigned short)(cvt_rs_bf16x2(0.0f, h, r) & 0xFFFFu));
  }
  __device__ static __nv_bfloat16 enc_host(double f, double shift) {
    return __double2bfloat16(f - shift);
  }
  __device__ static double dec_host(__nv_bfloat16 v, double shift) {
    return (double)__bfloat162float(v) + shift;
  }
};

// rho_s as the step uses it: the FP32 value of the shift density, so that the
// FP64 shift w_i rho_s of set-up and read-out matches the step's arithmetic.
__host__ __device__ inline double storage_rho_s(double rho_s) { return (double)(float)rho_s; }

constexpr int kMaxQ = 21;

// Random bits for stochastic rounding, drawn from a counter: one 32-bit word
// per (node pair, row, step) by the "lowbias32" integer hash (C. Wellons,
// hash-prospector) of a linear key, then one word per population i as the
// product with an odd multiplier (the splitmix64 output function of i + 1,
// made odd).  A paired encode gives the word to one conversion (first node:
// the low bits, see cvt_rs_f16x2); a one-node encode uses its low bits.
__host__ __device__ constexpr uint32_t sr_multiplier(int i) {
  uint64_t z = (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (uint32_t)z | 1u;
}

__device__ __forceinline__ uint32_t sr_hash(uint32_t x, uint32_t y, uint32_t step) {
  uint32_t h = x * 0x9E3779B1u + y * 0x85EBCA77u + step * 0xC2B2AE3Du;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return h;
}

// Ghost widths of the padded population layout.  x: at least 2R columns (the
// halo node's own pull) rounded up to 16 bytes so that every TMA box starts
// on a 16-byte boundary; y: 2R rows.
template <typename S, int R> __host__ __device__ constexpr int ghost_x() {
  return ((2 * R * (int)sizeof(S) + 15) / 16) * 16 / (int)sizeof(S);
}
template <int R> __host__ __device__ constexpr int ghost_y() { return 2 * R; }

// ---------------------------------------------------------------------------
// Run-time parameters of the update (compute precision T).
// ---------------------------------------------------------------------------
template <typename T> struct Physics {
  T omega;           // 1 / tau
  T one_m_omega;     // 1 - 1 / tau
  T G;               // fluid-fluid coupling in F_FF = -G psi sum w psi r
  T rho0;            // exponential psi scale
  T inv_rho0;        // 1 / rho0
  T exp2_scale;      // -log2(e) / rho0: exp(-rho / rho0) = 2^(rho exp2_scale)
  T eos_tv, eos_tu, eos_tl, eos_r1, eos_r2, eos_p1, eos_p2;
  T bfx, bfy;        // body-force density
  T rho_s;           // FP16S / BF16S shift density (stored h_i = sigma (f_i - w_i rho_s))
  T neg_omega_rho_s; // -rho_s / tau: the shift's share of the collision of h
  int32_t psi_kind;  // 0 exp, 1 EOS
  int32_t project;   // projection step on/off
};

template <typename T> struct WallFields {
  const T* phie;          // phi_S^epsilon            [ny][nx]
  const T* sx;            // S = sum_i w_i psi_FS(x + r_i) r_i
  const T* sy;
  const T* uwx;           // wall velocity (nullable)
  const T* uwy;
  int32_t active;         // 0: no wall at all; else per-(row, 32-column chunk) flags
                          // (uint32 [ny][nchunk_pad], non-zero where any wall term is
                          // non-zero) arrive by TMA with each row
};

template <typename T> __device__ __forceinline__ T t_exp(T v);
template <> __device__ __forceinline__ double t_exp<double>(double v) { return exp(v); }
template <> __device__ __forceinline__ float t_exp<float>(float v) { return expf(v); }
// 1 / rho.  FP64 divides exactly (quotients then divide, like the oracle);
// FP32 arithmetic: the hardware reciprocal (PTX rcp.approx.ftz.f32, at most
// 1 ulp from the correctly rounded value).
template <typename T> __device__ __forceinline__ T t_rcp(T v);
template <> __device__ __forceinline__ double t_rcp<double>(double v) { return 1.0 / v; }
template <> __device__ __forceinline__ float t_rcp<float>(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
// 1 / rho as the step uses it for storage S.  FP32 storage takes the correctly
// rounded reciprocal: the approximate one errs to one side more often than the
// other, and on an interface that bias in u = j / rho accumulates over the
// steps (on the 128x64 drop it doubles the density error after 1000 steps; a
// float32 restatement shows the same 2x from a one-ulp bias).  The FP32
// step is bound by HBM, so the few extra instructions cost nothing; 16-bit
// storage rounds far more coarsely and keeps the cheaper approximation.
template <typename S, typename T> __device__ __forceinline__ T rcp_node(T v) {
  if constexpr (std::is_same<S, float>::value) return __frcp_rn(v);
  else return t_rcp<T>(v);
}
template <typename T> __device__ __forceinline__ T t_fma(T a, T b, T c);
template <> __device__ __forceinline__ double t_fma<double>(double a, double b, double c) {
  return fma(a, b, c);
}
template <> __device__ __forceinline__ float t_fma<float>(float a, float b, float c) {
  return fmaf(a, b, c);
}
template <typename T> __device__ __forceinline__ T t_sqrt(T v);
template <> __device__ __forceinline__ double t_sqrt<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float t_sqrt<float>(float v) { return sqrtf(v); }

// 2^x by the hardware base-2 exponential (PTX ex2.approx.ftz.f32: a few
// units in the last place over the range used here).
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Exponential psi with FAST arithmetic: rho0 (1 - exp(-rho / rho0)) as
// rho0 - rho0 2^(rho c), c = -log2(e) / rho0, from the identity
// exp(y) = 2^(y log2 e).  One product, one hardware exponential and one fused
// multiply-add; about 2e-7 relative for the densities of a liquid-vapour
// system.  Used with 16-bit storage, whose rounding is about 2^-11 of a
// stored deviation; FP32 and FP64 storage keep expf / exp.
__device__ __forceinline__ float psi_exp_fast(float rho, float exp2_scale, float rho0) {
  return fmaf(ex2_approx(rho * exp2_scale), -rho0, rho0);
}

// psi(rho): exponential (Shan-Chen) or sqrt(2 [rho theta - p_EOS(rho)]) with the
// piecewise-linear Eq. EOS.  KIND: the kind if known at compile time (0
// exponential, 1 EOS), else -1 (P.psi_kind decides).  FAST: psi_exp_fast for
// the exponential kind (FP32 arithmetic).
template <int Q, typename T, int KIND = -1, bool FAST = false>
__device__ __forceinline__ T pseudo_potential(const Physics<T>& P, T rho) {
  if (KIND == 0 || (KIND < 0 && P.psi_kind == 0)) {
    if constexpr (FAST && sizeof(T) == 4) return psi_exp_fast(rho, P.exp2_scale, P.rho0);
    // FP64 divides like the oracle; FP32 multiplies by the reciprocal (exact
    // for the usual rho0 = 1).
    const T arg = sizeof(T) == 8 ? -rho / P.rho0 : -rho * P.inv_rho0;
    return P.rho0 * (T(1) - t_exp<T>(arg));
  }
  constexpr T theta = T(Lattice<Q>::THETA);
  T p;
  // Explicit fused operations: the same rounding in every kernel.
  if (rho <= P.eos_r1)
    p = rho * P.eos_tv;
  else if (rho <= P.eos_r2)
    p = t_fma<T>(rho - P.eos_r1, P.eos_tu, P.eos_p1);
  else
    p = t_fma<T>(rho - P.eos_r2, P.eos_tl, P.eos_p2);
  T arg = T(2) * t_fma<T>(rho, theta, -p);
  return t_sqrt<T>(arg > T(0) ? arg : T(0));
}

// c * v for a lattice coefficient c known at compile time: 0, +-v or c v
// (a product with zero is dropped; only the sign of a zero result can differ).
template <int C, typename T> __device__ __forceinline__ T cmul(T v) {
  if constexpr (C == 0) return T(0);
  else if constexpr (C == 1) return v;
  else if constexpr (C == -1) return -v;
  else return T(C) * v;
}
// c_x u_x + c_y u_y with compile-time c.
template <int CX, int CY, typename T> __device__ __forceinline__ T cdot(T ux, T uy) {
  if constexpr (CX == 0) return cmul<CY>(uy);
  else if constexpr (CY == 0) return cmul<CX>(ux);
  else return cmul<CX>(ux) + cmul<CY>(uy);
}

// Exact reciprocal constants of the equilibrium for each lattice.
template <int Q> struct EqConst;
template <> struct EqConst<9> {
  static constexpr double inv_theta = 3.0, inv_2theta2 = 4.5, inv_2theta = 1.5;
};
template <> struct EqConst<21> {
  static constexpr double inv_theta = 1.5, inv_2theta2 = 1.125, inv_2theta = 0.75;
};

// f_i^eq = w_i rho [1 + c.u / theta + (c.u)^2 / (2 theta^2) - u^2 / (2 theta)]
template <int Q, int I, typename T>
__device__ __forceinline__ T feq_c(T rho, T ux, T uy, T usq_term) {
  using L = Lattice<Q>;
  using E = EqConst<Q>;
  const T cu = cdot<L::cx(I), L::cy(I), T>(ux, uy);
  return T(L::w(I)) * rho * (T(1) + cu * T(E::inv_theta) + cu * cu * T(E::inv_2theta2) - usq_term);
}
template <int Q, typename T>
__device__ __forceinline__ T feq(int i, T rho, T ux, T uy, T usq_term) {
  using L = Lattice<Q>;
  using E = EqConst<Q>;
  const T cu = T(L::cx(i)) * ux + T(L::cy(i)) * uy;
  return T(L::w(i)) * rho * (T(1) + cu * T(E::inv_theta) + cu * cu * T(E::inv_2theta2) - usq_term);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1.
template <int I, int N, typename F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// Projection step (Sec. II, after Eq. f2): f_i <- w_i [rho + j.c_i / theta
//   + (Pi - rho theta I):(c_i c_i - theta I) / (2 theta^2)], Pi = sum f c c.
template <int Q, typename T>
__device__ __forceinline__ void project(T (&f)[Q], T rho, T jx, T jy) {
  using L = Lattice<Q>;
  using E = EqConst<Q>;
  constexpr T theta = T(L::THETA);
  T pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const T cx = T(L::cx(i)), cy = T(L::cy(i));
    pxx += f[i] * (cx * cx);
    pxy += f[i] * (cx * cy);
    pyy += f[i] * (cy * cy);
  }
  const T axx = pxx - rho * theta, ayy = pyy - rho * theta;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const T cx = T(L::cx(i)), cy = T(L::cy(i));
    const T contr = axx * (cx * cx - theta) + T(2) * pxy * (cx * cy) + ayy * (cy * cy - theta);
    f[i] = T(L::w(i)) * (rho + (jx * cx + jy * cy) * T(E::inv_theta) + contr * T(E::inv_2theta2));
  }
}


// a / b: FP64 divides (the oracle's rounding); FP32 multiplies by a reciprocal
// computed once per node.
template <typename T> __device__ __forceinline__ T div_rho(T a, T b, T inv_b);
template <> __device__ __forceinline__ double div_rho<double>(double a, double b, double) {
  return a / b;
}
template <> __device__ __forceinline__ float div_rho<float>(float a, float, float inv_b) {
  return a * inv_b;
}

// rho and j in table order.
template <int Q, typename T>
__device__ __forceinline__ void node_moments(const T (&f)[Q], T& rho, T& jx, T& jy) {
  using L = Lattice<Q>;
  rho = f[0];
  jx = T(L::cx(0)) * f[0];
  jy = T(L::cy(0)) * f[0];
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    rho += f[i];
    if (L::cx(i) == 1) jx += f[i];
    else if (L::cx(i) == -1) jx -= f[i];
    else if (L::cx(i) != 0) jx += T(L::cx(i)) * f[i];
    if (L::cy(i) == 1) jy += f[i];
    else if (L::cy(i) == -1) jy -= f[i];
    else if (L::cy(i) != 0) jy += T(L::cy(i)) * f[i];
  }
}

// Total force on a node (Eqs. force_SC, force_SC_FS, wall_shift):
//   F = F_FF + rho S + rho phi^eps (U_wall - u - F_FF / rho) + body force.
// sfx, sfy: sum_i w_i psi(x + r_i) r_i; wall terms only when has_wall.
template <typename T>
__device__ __forceinline__ void node_force(const Physics<T>& P, T rho, T ux, T uy, T psi_c,
                                           T sfx, T sfy, bool has_wall, T phie, T Sx, T Sy,
                                           T uwx, T uwy, T inv_rho, T& Fx, T& Fy) {
  const T mg = -P.G * psi_c;
  const T ffx = mg * sfx;
  const T ffy = mg * sfy;
  Fx = ffx;
  Fy = ffy;
  if (has_wall) {
    const T flx = rho * Sx, fly = rho * Sy;
    const T rp = rho * phie;
    const T dfx = rp * (uwx - ux - div_rho<T>(ffx, rho, inv_rho));
    const T dfy = rp * (uwy - uy - div_rho<T>(ffy, rho, inv_rho));
    Fx = ((ffx + flx) + dfx);
    Fy = ((ffy + fly) + dfy);
  }
  Fx += P.bfx;
  Fy += P.bfy;
}

// Index of the velocity opposite to c_i (compile time).
template <int Q> __host__ __device__ constexpr int opposite(int i) {
  using L = Lattice<Q>;
  for (int j = 0; j < Q; ++j)
    if (L::cx(j) == -L::cx(i) && L::cy(j) == -L::cy(i)) return j;
  return i;
}

// EDM-BGK collision (Eq. BE-BGK with the exact-difference forcing):
//   f_post = f - (f - f^eq(rho, u)) / tau + [f^eq(rho, u*) - f^eq(rho, u)]
//          = g f + f^eq(u*) - g f^eq(u),          g = 1 - 1/tau, omega = 1/tau.
// With the second-order equilibrium this splits, for each pair of opposite
// velocities +-c, into a part even and a part odd in c:
//   f_post(+-c) = g f(+-c) + S +- A,
//   S = w rho [omega - B + ((c.u*)^2 - g (c.u)^2) / (2 theta^2)],
//   A = w rho c.(u* - g u) / theta,   B = (u*^2 - g u^2) / (2 theta),
// and f_post(rest) = g f(rest) + w_rest rho (omega - B).  This is the same
// update evaluated with about half the arithmetic of two full equilibria.
//
// With FP32 arithmetic the rest population is then taken from the mass
// balance sum_i f_i^post = rho, which the update satisfies identically:
// evaluating every term in single precision otherwise leaves a rounding bias
// in the node's mass (of order 1e-7 rho per step, correlated in space and
// time) that accumulates into a visible density drift at interfaces.
template <int Q, typename T>
__device__ __forceinline__ void node_collide(const Physics<T>& P, T (&f)[Q], T rho, T ux, T uy,
                                             T usx, T usy) {
  using E = EqConst<Q>;
  using L = Lattice<Q>;
  const T g = P.one_m_omega;
  const T ax = usx - g * ux, ay = usy - g * uy;
  const T Bt = (usx * usx + usy * usy - g * (ux * ux + uy * uy)) * T(E::inv_2theta);
  const T wB = P.omega - Bt;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr int j = opposite<Q>(i);
    if constexpr (i == L::REST) {
      f[i] = g * f[i] + T(L::w(i)) * rho * wB;
    } else if constexpr (i < j) {
      const T cs = cdot<L::cx(i), L::cy(i), T>(usx, usy);
      const T cu = cdot<L::cx(i), L::cy(i), T>(ux, uy);
      const T ca = cdot<L::cx(i), L::cy(i), T>(ax, ay);
      const T wr = T(L::w(i)) * rho;
      const T t = cs * cs - g * (cu * cu);
      const T S = wr * (wB + t * T(E::inv_2theta2));
      const T A = wr * (ca * T(E::inv_theta));
      const T fi = g * f[i] + (S + A);
      const T fj = g * f[j] + (S - A);
      f[i] = fi;
      f[j] = fj;
    }
  });
  if constexpr (sizeof(T) == 4) {
    T moving = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (i != L::REST) moving += f[i];
    f[L::REST] = rho - moving;
  }
}

}  // namespace lbm
