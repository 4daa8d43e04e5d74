// Set-up and read-out kernels: population encode / decode between the FP64
// user layout [Q][ny][nx] (post-streaming f_i(x, t)) and the padded device
// layout (post-collision f_i^post at the emitting node, with periodic ghost
// images), the equilibrium initialiser (Eq. feqc), the wall-field preparation
// (phi_S^eps and S = sum_i w_i psi_FS(x + r_i) r_i, Eqs. force_SC_FS and
// pseudopotential), deterministic FP64 reductions, and one pass of the
// Appendix's recursive wall filter (Eq. iteration).
#include <cuda_runtime.h>

#include "launch.cuh"

namespace lbm {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Writes value v of population plane i for node (x, y) to the node and to every
// periodic image of it inside the ghost frame.
template <typename S, int GX, int GY>
__device__ inline void store_images(S* buf, int64_t plane, int64_t pitch, int i, int x, int y,
                                    int nx, int ny, S v) {
  int xa = x;
  while (xa - nx >= -GX) xa -= nx;
  int ya = y;
  while (ya - ny >= -GY) ya -= ny;
  for (int ym = ya; ym < ny + GY; ym += ny)
    for (int xm = xa; xm < nx + GX; xm += nx)
      buf[i * plane + (int64_t)(ym + GY) * pitch + (xm + GX)] = v;
}

// Device layout holds P_i(x) = f_i(x + c_i) (the value that streams into x + c_i).
template <int Q, typename S>
__global__ void encode_kernel(const double* __restrict__ f, S* __restrict__ buf, int nx, int ny,
                              int64_t pitch, int64_t plane, double rho_s) {
  using L = Lattice<Q>;
  constexpr int R = L::R;
  constexpr int GX = ghost_x<S, R>(), GY = ghost_y<R>();
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (int64_t)nx * ny) return;
  const int x = (int)(n % nx), y = (int)(n / nx);
  const int64_t N = (int64_t)nx * ny;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int xs = wrap(x + L::cx(i), nx), ys = wrap(y + L::cy(i), ny);
    const double v = f[i * N + (int64_t)ys * nx + xs];
    const S e = Codec<S>::enc_host(v, L::w(i) * rho_s);
    store_images<S, GX, GY>(buf, plane, pitch, Planes<Q>::template plane<i>, x, y, nx, ny, e);
  });
}

template <int Q, typename S>
__global__ void equilibrium_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                                   const double* __restrict__ uy, const double* __restrict__ dfi,
                                   S* __restrict__ buf, int nx, int ny, int64_t pitch,
                                   int64_t plane, double rho_s) {
  using L = Lattice<Q>;
  using E = EqConst<Q>;
  constexpr int R = L::R;
  constexpr int GX = ghost_x<S, R>(), GY = ghost_y<R>();
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (int64_t)nx * ny) return;
  const int x = (int)(n % nx), y = (int)(n / nx);
  const int64_t N = (int64_t)nx * ny;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int64_t m = (int64_t)wrap(y + L::cy(i), ny) * nx + wrap(x + L::cx(i), nx);
    const double r = rho[m], vx = ux[m], vy = uy[m];
    const double usq = (vx * vx + vy * vy) * E::inv_2theta;
    double v = feq<Q, double>(i, r, vx, vy, usq);
    if (dfi) v = v + dfi[i * N + m];
    const S e = Codec<S>::enc_host(v, L::w(i) * rho_s);
    store_images<S, GX, GY>(buf, plane, pitch, Planes<Q>::template plane<i>, x, y, nx, ny, e);
  });
}

template <int Q, typename S>
__global__ void decode_kernel(const S* __restrict__ buf, double* __restrict__ f, int nx, int ny,
                              int64_t pitch, int64_t plane, double rho_s) {
  using L = Lattice<Q>;
  constexpr int R = L::R;
  constexpr int GX = ghost_x<S, R>(), GY = ghost_y<R>();
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (int64_t)nx * ny) return;
  const int x = (int)(n % nx), y = (int)(n / nx);
  const int64_t N = (int64_t)nx * ny;
  static_for<0, Q>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    // f_i(x) = P_i(x - c_i); the ghost frame makes the source in-bounds.
    const int64_t src = Planes<Q>::template plane<i> * plane +
                        (int64_t)(y - L::cy(i) + GY) * pitch + (x - L::cx(i) + GX);
    f[i * N + n] = Codec<S>::dec_host(buf[src], L::w(i) * rho_s);
  });
}

// phi_S^eps, S(x) = sum_i w_i psi_FS(x + r_i) r_i with psi_FS = G_A psi_A - G_R psi_R
// (table order, FP64), optional wall velocity; then converted to T.
template <int Q, typename T>
__global__ void wall_prepare_kernel(const double* __restrict__ phi, const double* __restrict__ psr,
                                    const double* __restrict__ psa, const double* __restrict__ uw,
                                    double G_R, double G_A, double eps, int nx, int ny,
                                    T* __restrict__ phie, T* __restrict__ sx, T* __restrict__ sy,
                                    T* __restrict__ uwx, T* __restrict__ uwy) {
  using L = Lattice<Q>;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = (int64_t)nx * ny;
  if (n >= N) return;
  const int x = (int)(n % nx), y = (int)(n / nx);
  double ax = 0.0, ay = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int64_t m = (int64_t)wrap(y + L::cy(i), ny) * nx + wrap(x + L::cx(i), nx);
    double pfs = 0.0;
    if (psa) pfs = pfs + G_A * psa[m];
    if (psr) pfs = pfs - G_R * psr[m];
    ax = ax + L::w(i) * pfs * L::cx(i);
    ay = ay + L::w(i) * pfs * L::cy(i);
  }
  double pe = 0.0;
  if (phi) pe = (eps == 1.0) ? phi[n] : pow(phi[n], eps);
  phie[n] = (T)pe;
  sx[n] = (T)ax;
  sy[n] = (T)ay;
  if (uwx) {
    uwx[n] = (T)uw[n];
    uwy[n] = (T)uw[N + n];
  }
}

// flags[y][c] = 1 when any of phi^eps, S_x, S_y is non-zero in columns
// 32c..32c+31 (0 in the padding chunks past nx).
template <typename T>
__global__ void wall_flags_kernel(const T* __restrict__ phie, const T* __restrict__ sx,
                                  const T* __restrict__ sy, int nx, int ny, int nchunk_pad,
                                  uint32_t* __restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nchunk_pad * ny) return;
  const int y = (int)(t / nchunk_pad), c = (int)(t % nchunk_pad);
  uint32_t any = 0;
  for (int x = 32 * c; x < min(nx, 32 * c + 32); ++x) {
    const int64_t n = (int64_t)y * nx + x;
    if (phie[n] != T(0) || sx[n] != T(0) || sy[n] != T(0)) any = 1;
  }
  flags[t] = any;
}

// Neumaier-compensated accumulate.
__device__ inline void neum_add(double& s, double& c, double v) {
  const double t = s + v;
  if (fabs(s) >= fabs(v))
    c += (s - t) + v;
  else
    c += (v - t) + s;
  s = t;
}

// Per-block compensated sums of up to three arrays, then a fixed-order tree.
__global__ void reduce3_kernel(const double* __restrict__ a, const double* __restrict__ b,
                               const double* __restrict__ c, int64_t n,
                               double* __restrict__ partials) {
  __shared__ double sh[3][2][kThreads];
  double s[3] = {0, 0, 0}, k[3] = {0, 0, 0};
  const double* src[3] = {a, b, c};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int q = 0; q < 3; ++q)
      if (src[q]) neum_add(s[q], k[q], src[q][i]);
  }
  for (int q = 0; q < 3; ++q) {
    sh[q][0][threadIdx.x] = s[q];
    sh[q][1][threadIdx.x] = k[q];
  }
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      for (int q = 0; q < 3; ++q) {
        double ss = sh[q][0][threadIdx.x], cc = sh[q][1][threadIdx.x];
        neum_add(ss, cc, sh[q][0][threadIdx.x + w]);
        cc += sh[q][1][threadIdx.x + w];
        sh[q][0][threadIdx.x] = ss;
        sh[q][1][threadIdx.x] = cc;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) {
      partials[(int64_t)blockIdx.x * 6 + 2 * q] = sh[q][0][0];
      partials[(int64_t)blockIdx.x * 6 + 2 * q + 1] = sh[q][1][0];
    }
  }
}

__global__ void reduce3_final_kernel(const double* __restrict__ partials, int nparts,
                                     double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < 3; ++q) {
    double s = 0.0, c = 0.0;
    for (int p = 0; p < nparts; ++p) {
      neum_add(s, c, partials[6 * p + 2 * q]);
      c += partials[6 * p + 2 * q + 1];
    }
    out[q] = s + c;
  }
}

// out[n] = sum_i f[i][n] in table order (rho of a population array).
__global__ void colsum_kernel(const double* __restrict__ f, int q, int64_t n,
                              double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s = f[t];
  for (int i = 1; i < q; ++i) s = s + f[(int64_t)i * n + t];
  out[t] = s;
}

// One pass of the Appendix filter: out = sum_i w_i g(x + r_i), reset to 1 on solid nodes.
template <int Q>
__global__ void filter_pass_kernel(const double* __restrict__ g, double* __restrict__ out,
                                   const uint8_t* __restrict__ solid, int nx, int ny) {
  using L = Lattice<Q>;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (int64_t)nx * ny) return;
  const int x = (int)(n % nx), y = (int)(n / nx);
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    acc = acc + L::w(i) * g[(int64_t)wrap(y + L::cy(i), ny) * nx + wrap(x + L::cx(i), nx)];
  out[n] = solid[n] ? 1.0 : acc;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

template <int Q, typename S>
cudaError_t launch_encode(const double* f, S* buf, int nx, int ny, int64_t pitch, int64_t plane,
                          double rho_s, cudaStream_t st) {
  encode_kernel<Q, S><<<blocks_for((int64_t)nx * ny), kThreads, 0, st>>>(f, buf, nx, ny, pitch,
                                                                         plane, rho_s);
  return cudaGetLastError();
}

template <int Q, typename S>
cudaError_t launch_equilibrium(const double* rho, const double* ux, const double* uy,
                               const double* dfi, S* buf, int nx, int ny, int64_t pitch,
                               int64_t plane, double rho_s, cudaStream_t st) {
  equilibrium_kernel<Q, S><<<blocks_for((int64_t)nx * ny), kThreads, 0, st>>>(
      rho, ux, uy, dfi, buf, nx, ny, pitch, plane, rho_s);
  return cudaGetLastError();
}

template <int Q, typename S>
cudaError_t launch_decode(const S* buf, double* f, int nx, int ny, int64_t pitch, int64_t plane,
                          double rho_s, cudaStream_t st) {
  decode_kernel<Q, S><<<blocks_for((int64_t)nx * ny), kThreads, 0, st>>>(buf, f, nx, ny, pitch,
                                                                         plane, rho_s);
  return cudaGetLastError();
}

template <int Q, typename T>
cudaError_t launch_wall_prepare(const double* phi, const double* psr, const double* psa,
                                const double* uw, double G_R, double G_A, double eps, int nx,
                                int ny, T* phie, T* sx, T* sy, T* uwx, T* uwy, uint32_t* flags,
                                int nchunk_pad, cudaStream_t st) {
  const int64_t N = (int64_t)nx * ny;
  wall_prepare_kernel<Q, T><<<blocks_for(N), kThreads, 0, st>>>(phi, psr, psa, uw, G_R, G_A, eps,
                                                                nx, ny, phie, sx, sy, uwx, uwy);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wall_flags_kernel<T><<<blocks_for((int64_t)nchunk_pad * ny), kThreads, 0, st>>>(
      phie, sx, sy, nx, ny, nchunk_pad, flags);
  return cudaGetLastError();
}

cudaError_t launch_reduce3(const double* a, const double* b, const double* c, int64_t n,
                           double* partials, int nparts, double* out, cudaStream_t st) {
  reduce3_kernel<<<nparts, kThreads, 0, st>>>(a, b, c, n, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce3_final_kernel<<<1, 32, 0, st>>>(partials, nparts, out);
  return cudaGetLastError();
}

cudaError_t launch_colsum(const double* f, int q, int64_t n, double* out_n, cudaStream_t st) {
  colsum_kernel<<<blocks_for(n), kThreads, 0, st>>>(f, q, n, out_n);
  return cudaGetLastError();
}

cudaError_t launch_filter_pass(int q, const double* g, double* out, const uint8_t* solid, int nx,
                               int ny, cudaStream_t st) {
  const int64_t N = (int64_t)nx * ny;
  if (q == 9)
    filter_pass_kernel<9><<<blocks_for(N), kThreads, 0, st>>>(g, out, solid, nx, ny);
  else
    filter_pass_kernel<21><<<blocks_for(N), kThreads, 0, st>>>(g, out, solid, nx, ny);
  return cudaGetLastError();
}

#define LBM_INSTANTIATE_AUX(Q, S)                                                               \
  template cudaError_t launch_encode<Q, S>(const double*, S*, int, int, int64_t, int64_t, double, \
                                           cudaStream_t);                                       \
  template cudaError_t launch_equilibrium<Q, S>(const double*, const double*, const double*,    \
                                                const double*, S*, int, int, int64_t, int64_t,  \
                                                double, cudaStream_t);                          \
  template cudaError_t launch_decode<Q, S>(const S*, double*, int, int, int64_t, int64_t, double, \
                                           cudaStream_t);

LBM_INSTANTIATE_AUX(9, double)
LBM_INSTANTIATE_AUX(9, float)
LBM_INSTANTIATE_AUX(9, __half)
LBM_INSTANTIATE_AUX(9, __nv_bfloat16)
LBM_INSTANTIATE_AUX(21, double)
LBM_INSTANTIATE_AUX(21, float)
LBM_INSTANTIATE_AUX(21, __half)
LBM_INSTANTIATE_AUX(21, __nv_bfloat16)

#define LBM_INSTANTIATE_WALL(Q, T)                                                            \
  template cudaError_t launch_wall_prepare<Q, T>(const double*, const double*, const double*, \
                                                 const double*, double, double, double, int,  \
                                                 int, T*, T*, T*, T*, T*, uint32_t*, int,      \
                                                 cudaStream_t);
LBM_INSTANTIATE_WALL(9, double)
LBM_INSTANTIATE_WALL(9, float)
LBM_INSTANTIATE_WALL(21, double)
LBM_INSTANTIATE_WALL(21, float)

}  // namespace lbm
