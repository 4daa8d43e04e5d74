// C ABI of the engine (include/lbm.h): context life cycle, device memory,
// TMA descriptors, launch-shape selection and dispatch over (lattice, storage).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <initializer_list>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/lbm.h"
#include "launch.cuh"

using namespace lbm;

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct lbm_ctx {
  lbm_params p{};
  int Q = 9, R = 1, GX = 0, GY = 0, esize = 4, W = 128, NS = 8;
  int64_t pitch = 0, rows = 0, plane = 0;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding the current state
  PopMaps tmap[2];       // population maps of buffer 0 and 1 (one per box depth)
  // wall (compute precision: double for FP64 storage, float otherwise)
  void* wall_phie = nullptr;
  void* wall_sx = nullptr;
  void* wall_sy = nullptr;
  void* wall_uwx = nullptr;
  void* wall_uwy = nullptr;
  uint32_t* wall_flags = nullptr;  // [ny][nchunk_pad]
  int nchunk_pad = 0;
  int flag_box = 0;                // flag words per TMA box (ConfigShape::FLAG_BOX)
  CUtensorMap flag_map;
  bool has_wall = false;
  uint32_t* d_status = nullptr;  // 256 bytes: word 0 status bits, words kRngWord.. step counter
  double* d_partials = nullptr;
  int nparts = 0;
  double* d_out3 = nullptr;
  cudaStream_t stream = nullptr;
  lbm_allocator alloc{};
  bool user_alloc = false;
  std::vector<void*> owned;
  std::string err;
  bool poisoned = false;
  bool has_state = false;
  int64_t steps = 0;
  double rho_s = 0.0;
  int tile_rows = 0, grid_x = 0, grid_y = 0;
  uint64_t version = 0;  // bumped whenever device pointers or parameters change
  uint64_t wait_ns = 2000000000ull;  // bound of every stage wait in the step kernels
  uint64_t stall_wait_ns = 0;        // test hook: armed stall for the next step
};

namespace {

// The two step-counter words of the stochastic rounding live in the status
// allocation (its own 64-byte line).
constexpr int kRngWord = 16;


thread_local std::string g_err;  // errors of calls without a context

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = msg;
    if (code == LBM_ECUDA) c->poisoned = true;
  } else {
    g_err = msg;
  }
  return code;
}

#define CK(ctx, ...)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (__VA_ARGS__);                                                     \
    if (e_ != cudaSuccess)                                                              \
      return fail((ctx), LBM_ECUDA, "%s failed: %s (%s:%d)", #__VA_ARGS__,                \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                          \
  } while (0)

void* dalloc(lbm_ctx* c, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->user_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->owned.push_back(p);
  return p;
}

void dfree(lbm_ctx* c, void* p) {
  if (!p) return;
  auto it = std::find(c->owned.begin(), c->owned.end(), p);
  if (it != c->owned.end()) c->owned.erase(it);
  if (c->user_alloc)
    c->alloc.free(p, c->alloc.user);
  else
    cudaFree(p);
}

// Scoped temporary device allocation.
struct Tmp {
  lbm_ctx* c;
  void* p;
  Tmp(lbm_ctx* c_, size_t bytes) : c(c_), p(bytes ? dalloc(c_, bytes) : nullptr) {}
  ~Tmp() {
    if (p) {
      cudaStreamSynchronize(c->stream);
      dfree(c, p);
    }
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

int guard(lbm_ctx* c) {
  if (!c) return fail(nullptr, LBM_EINVAL, "null context");
  if (c->poisoned) return fail(c, LBM_ESTATE, "context poisoned by an earlier CUDA error: %s", c->err.c_str());
  return LBM_OK;
}

// --- dispatch over (lattice, storage) ---------------------------------------
template <typename F> int dispatch(int Q, int storage, F&& fn) {
  switch (Q * 10 + storage) {
    case 90: return fn.template operator()<9, double>();
    case 91: return fn.template operator()<9, float>();
    case 92: return fn.template operator()<9, __half>();
    case 93: return fn.template operator()<9, __nv_bfloat16>();
    case 210: return fn.template operator()<21, double>();
    case 211: return fn.template operator()<21, float>();
    case 212: return fn.template operator()<21, __half>();
    case 213: return fn.template operator()<21, __nv_bfloat16>();
  }
  return LBM_EINVAL;
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
  static EncodeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeFn>(p);
  }();
  return fn;
}

template <typename S> CUtensorMapDataType tma_type();
template <> CUtensorMapDataType tma_type<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <> CUtensorMapDataType tma_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> CUtensorMapDataType tma_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <> CUtensorMapDataType tma_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

template <int Q, typename S> int make_tmap(lbm_ctx* c, int which) {
  using Sh = ConfigShape<Q, S>;
  EncodeFn enc = get_encode();
  if (!enc) return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
  cuuint64_t dims[3] = {(cuuint64_t)(c->p.nx + 2 * Sh::GX), (cuuint64_t)c->rows, (cuuint64_t)Q};
  cuuint64_t strides[2] = {(cuuint64_t)(c->pitch * sizeof(S)),
                           (cuuint64_t)(c->plane * sizeof(S))};
  cuuint32_t estr[3] = {1, 1, 1};
  c->tmap[which] = PopMaps{};
  for (int k = 0; k < Sh::NMAP; ++k) {
    // One box: a row of BW elements of Sh::kTab.depth[k] consecutive planes.
    cuuint32_t box[3] = {(cuuint32_t)Sh::BW, 1, (cuuint32_t)Sh::kTab.depth[k]};
    CUresult r = enc(&c->tmap[which].m[k], tma_type<S>(), 3, c->buf[which], dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  }
  return LBM_OK;
}

// Rows per CTA segment.  Measured on GB300 (8192x4096 D2Q9 sweep): short
// segments run fastest -- many waves of short CTAs keep the concurrently
// active tiles in a compact band of rows and balance the SMs dynamically; with
// adjacent segments marching in opposite directions the 2R halo rows they
// share are pulled at about the same time and the second pull hits in L2.
// FP32 is fastest at 4-5 rows (0.3640 ms against 0.3668 at 6, 0.3722 at 8 and
// 0.3775 at 3), 16-bit storage near 24, FP64 near 64.  Small
// lattices get shorter segments so that the grid still covers at least two
// waves of resident CTAs.
int choose_tile_rows(int nx, int ny, int W, int esize, int R, int ctas_per_sm, int num_sms) {
  const int gx = (nx + W - 1) / W;
  const int64_t slots = (int64_t)std::max(1, ctas_per_sm) * num_sms;
  int L = esize == 2 ? 24 : (esize == 4 ? 4 : 64);
  if (R > 1) L = std::max(L, 16 * R);
  while (L > 4 && (int64_t)gx * ((ny + L - 1) / L) < 2 * slots) L /= 2;
  return std::max(1, std::min(L, ny));
}

template <int Q, typename S> int setup_layout(lbm_ctx* c) {
  using Sh = ConfigShape<Q, S>;
  c->Q = Q;
  c->R = Sh::R;
  c->GX = Sh::GX;
  c->GY = Sh::GY;
  c->esize = (int)sizeof(S);
  c->W = StepConfig<Q, S>::W;
  c->flag_box = Sh::FLAG_BOX;
  c->NS = StepConfig<Q, S>::NS;
  c->pitch = ((int64_t)(c->p.nx + 2 * Sh::GX) + 31) / 32 * 32;
  c->rows = c->p.ny + 2 * Sh::GY;
  c->plane = c->pitch * c->rows;
  const size_t bytes = (size_t)c->plane * Q * sizeof(S);
  for (int b = 0; b < 2; ++b) {
    c->buf[b] = dalloc(c, bytes);
    if (!c->buf[b]) return fail(c, LBM_ENOMEM, "population buffer of %zu bytes", bytes);
    CK(c, cudaMemsetAsync(c->buf[b], 0, bytes, c->stream));
    int rc = make_tmap<Q, S>(c, b);
    if (rc) return rc;
  }
  int dev = 0, sms = 0;
  CK(c, cudaGetDevice(&dev));
  CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int cps = step_ctas_per_sm<Q, S>();
  if (cps <= 0) {
    cudaError_t e = cudaGetLastError();
    return fail(c, LBM_ECUDA, "step kernel cannot be resident (%s)", cudaGetErrorString(e));
  }
  c->tile_rows = c->p.tile_rows > 0 ? std::min(c->p.tile_rows, c->p.ny)
                                    : choose_tile_rows(c->p.nx, c->p.ny, c->W, c->esize, c->R, cps, sms);
  c->grid_x = (c->p.nx + c->W - 1) / c->W;
  c->grid_y = (c->p.ny + c->tile_rows - 1) / c->tile_rows;
  return LBM_OK;
}

template <typename T> Physics<T> make_physics(const lbm_ctx* c) {
  const lbm_params& p = c->p;
  Physics<T> P;
  P.omega = (T)(1.0 / p.tau);
  P.one_m_omega = (T)(1.0 - 1.0 / p.tau);
  P.G = (T)p.G;
  P.rho0 = (T)p.rho0;
  P.inv_rho0 = (T)(1.0 / p.rho0);
  P.exp2_scale = (T)(-1.4426950408889634 / p.rho0);  // -log2(e) / rho0
  P.eos_tv = (T)p.eos_theta_v;
  P.eos_tu = (T)p.eos_theta_u;
  P.eos_tl = (T)p.eos_theta_l;
  P.eos_r1 = (T)p.eos_rho1;
  P.eos_r2 = (T)p.eos_rho2;
  const double p1 = p.eos_rho1 * p.eos_theta_v;
  const double p2 = p.eos_rho1 * p.eos_theta_v + (p.eos_rho2 - p.eos_rho1) * p.eos_theta_u;
  P.eos_p1 = (T)p1;
  P.eos_p2 = (T)p2;
  P.bfx = (T)p.body_force[0];
  P.bfy = (T)p.body_force[1];
  P.rho_s = (T)c->rho_s;
  P.neg_omega_rho_s = (T)(-c->rho_s / p.tau);
  P.psi_kind = p.psi_kind;
  P.project = p.project;
  return P;
}

// Step arguments for a pass that reads the current buffer of c.
// Step arguments for a pass that reads buffer `src` of c (the current one for
// run_pass; either for the batch descriptors).
template <int Q, typename S>
StepArgs<typename Codec<S>::T, S> make_args(const lbm_ctx* c, int src, S* fout, double* o_rho,
                                            double* o_ux, double* o_uy, int momentum) {
  using T = typename Codec<S>::T;
  StepArgs<T, S> a{};
  a.phys = make_physics<T>(c);
  a.wall.phie = static_cast<const T*>(c->wall_phie);
  a.wall.sx = static_cast<const T*>(c->wall_sx);
  a.wall.sy = static_cast<const T*>(c->wall_sy);
  a.wall.uwx = static_cast<const T*>(c->wall_uwx);
  a.wall.uwy = static_cast<const T*>(c->wall_uwy);
  a.wall.active = c->has_wall ? 1 : 0;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.pitch = (int32_t)c->pitch;
  a.tile_rows = c->tile_rows;
  a.plane = c->plane;
  a.fout = fout;
  a.out_rho = o_rho;
  a.out_ux = o_ux;
  a.out_uy = o_uy;
  a.momentum = momentum;
  a.status = c->d_status;
  a.wait_ns = c->stall_wait_ns ? c->stall_wait_ns : c->wait_ns;
  a.extra_tx = c->stall_wait_ns ? 16u : 0u;
  a.rng = c->d_status + kRngWord;
  a.rng_idx = src;
  a.stochastic = c->p.rounding == LBM_ROUND_STOCHASTIC ? 1 : 0;
  return a;
}

template <int Q, typename S>
int run_pass(lbm_ctx* c, int mode, double* o_rho, double* o_ux, double* o_uy, int momentum,
             S* fout) {
  const auto a = make_args<Q, S>(c, c->cur, fout, o_rho, o_ux, o_uy, momentum);
  // Without walls the flag map is never read; the population map stands in.
  const CUtensorMap& fm = c->has_wall ? c->flag_map : c->tmap[c->cur].m[0];
  CK(c, launch_step<Q, S>(c->tmap[c->cur], fm, a, dim3(c->grid_x, c->grid_y), c->stream, mode));
  return LBM_OK;
}

int check_params(const lbm_params* p) {
  if (!p) return fail(nullptr, LBM_EINVAL, "null params");
  if (p->nx < 1 || p->ny < 1) return fail(nullptr, LBM_EINVAL, "lattice size %dx%d", p->nx, p->ny);
  if ((int64_t)p->nx * p->ny > (int64_t)1 << 31)
    return fail(nullptr, LBM_EINVAL, "lattice of %lld nodes exceeds 2^31", (long long)p->nx * p->ny);
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D2Q21)
    return fail(nullptr, LBM_EINVAL, "lattice %d", p->lattice);
  if (p->storage < LBM_FP64 || p->storage > LBM_BF16S)
    return fail(nullptr, LBM_EINVAL, "storage %d", p->storage);
  if (p->psi_kind != LBM_PSI_EXP && p->psi_kind != LBM_PSI_EOS)
    return fail(nullptr, LBM_EINVAL, "psi_kind %d", p->psi_kind);
  if (!(p->tau > 0.5) || !std::isfinite(p->tau))
    return fail(nullptr, LBM_EINVAL, "tau must be > 0.5 (got %g)", p->tau);
  if (p->psi_kind == LBM_PSI_EXP && !(p->rho0 > 0.0))
    return fail(nullptr, LBM_EINVAL, "rho0 must be > 0");
  if (p->psi_kind == LBM_PSI_EOS && !(p->eos_rho1 < p->eos_rho2))
    return fail(nullptr, LBM_EINVAL, "EOS knots must satisfy rho1 < rho2");
  if (p->check_every < 0 || p->tile_rows < 0) return fail(nullptr, LBM_EINVAL, "negative count");
  if (p->rounding != LBM_ROUND_STOCHASTIC && p->rounding != LBM_ROUND_NEAREST)
    return fail(nullptr, LBM_EINVAL, "rounding %d", p->rounding);
  return LBM_OK;
}

// Shift for FP16S / BF16S: the configured value, else the mean of rho.
int set_shift_from_rho(lbm_ctx* c, const double* d_rho) {
  if (c->p.storage != LBM_FP16S && c->p.storage != LBM_BF16S) {
    c->rho_s = 0.0;
    return LBM_OK;
  }
  if (c->p.shift_rho > 0.0) {
    c->rho_s = storage_rho_s(c->p.shift_rho);
    return LBM_OK;
  }
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  CK(c, launch_reduce3(d_rho, nullptr, nullptr, N, c->d_partials, c->nparts, c->d_out3, c->stream));
  double h[3];
  CK(c, cudaMemcpyAsync(h, c->d_out3, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->rho_s = storage_rho_s(h[0] / (double)N);
  return LBM_OK;
}

}  // namespace

// Sets the context-free error text (used by entry points defined in other
// translation units; not exported).
void lbmi_set_error(const char* msg) { g_err = msg ? msg : ""; }

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

int lbm_params_default(lbm_params* p) {
  if (!p) return fail(nullptr, LBM_EINVAL, "null params");
  std::memset(p, 0, sizeof *p);
  p->nx = 128;
  p->ny = 64;
  p->lattice = LBM_D2Q9;
  p->storage = LBM_FP32;
  p->psi_kind = LBM_PSI_EXP;
  p->tau = 1.0;
  p->G = -5.5;
  p->rho0 = 1.0;
  const double th = 1.0 / 3.0;
  p->eos_theta_v = 0.25 * th;
  p->eos_theta_u = -0.25 * th;
  p->eos_theta_l = 1.0 * th;
  p->eos_rho1 = 0.222;
  p->eos_rho2 = 0.869;
  return LBM_OK;
}

int lbm_create(const lbm_params* p, const lbm_allocator* a, void* cuda_stream, lbm_ctx** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "null output pointer");
  *out = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  if (a && (!a->alloc || !a->free)) return fail(nullptr, LBM_EINVAL, "allocator without alloc/free");
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation");
  c->p = *p;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (a) {
    c->alloc = *a;
    c->user_alloc = true;
  }
  rc = dispatch(p->lattice, p->storage, [&]<int Q, typename S>() { return setup_layout<Q, S>(c); });
  if (rc == LBM_OK) {
    c->d_status = static_cast<uint32_t*>(dalloc(c, 256));
    c->nparts = kReduceParts;
    c->d_partials = static_cast<double*>(dalloc(c, sizeof(double) * 6 * c->nparts));
    c->d_out3 = static_cast<double*>(dalloc(c, 256));
    if (!c->d_status || !c->d_partials || !c->d_out3)
      rc = fail(c, LBM_ENOMEM, "status / reduction buffers");
    else if (cudaMemsetAsync(c->d_status, 0, 256, c->stream) != cudaSuccess)
      rc = fail(c, LBM_ECUDA, "cudaMemsetAsync status");
  }
  if (rc != LBM_OK) {
    g_err = c->err;
    lbm_destroy(c);
    return rc;
  }
  *out = c;
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx* c, void* cuda_stream) {
  int rc = guard(c);
  if (rc) return rc;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->version += 1;
  return LBM_OK;
}

int lbm_set_wall(lbm_ctx* c, const double* phi_s, const double* psi_r, const double* psi_a,
                 double G_R, double G_A, double epsilon, const double* u_wall) {
  int rc = guard(c);
  if (rc) return rc;
  if (!(epsilon > 0.0) || !std::isfinite(G_R) || !std::isfinite(G_A))
    return fail(c, LBM_EINVAL, "wall parameters (epsilon %g, G_R %g, G_A %g)", epsilon, G_R, G_A);
  const int nx = c->p.nx, ny = c->p.ny;
  const int64_t N = (int64_t)nx * ny;
  const size_t tsz = c->p.storage == LBM_FP64 ? sizeof(double) : sizeof(float);
  if (!c->wall_phie) {
    // one uint32 flag per (row, 32-column chunk); rows padded to 16 bytes so
    // that each strip's flag words are one aligned TMA box
    c->nchunk_pad = ((nx + 31) / 32 + 3) / 4 * 4;
    c->wall_phie = dalloc(c, N * tsz);
    c->wall_sx = dalloc(c, N * tsz);
    c->wall_sy = dalloc(c, N * tsz);
    c->wall_flags = static_cast<uint32_t*>(dalloc(c, (size_t)c->nchunk_pad * ny * 4));
    if (!c->wall_phie || !c->wall_sx || !c->wall_sy || !c->wall_flags)
      return fail(c, LBM_ENOMEM, "wall fields");
    EncodeFn enc = get_encode();
    if (!enc) return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)c->nchunk_pad, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)c->nchunk_pad * 4};
    cuuint32_t box[2] = {(cuuint32_t)c->flag_box, 1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&c->flag_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, c->wall_flags, dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, LBM_ECUDA, "flag tensor map (%d)", (int)r);
  }
  if (u_wall && !c->wall_uwx) {
    c->wall_uwx = dalloc(c, N * tsz);
    c->wall_uwy = dalloc(c, N * tsz);
    if (!c->wall_uwx || !c->wall_uwy) return fail(c, LBM_ENOMEM, "wall velocity");
  }
  Tmp stage(c, (size_t)N * 5 * sizeof(double));
  if (!stage.p) return fail(c, LBM_ENOMEM, "wall staging");
  double* d = stage.as<double>();
  const double* src[4] = {phi_s, psi_r, psi_a, u_wall};
  double* dst[4] = {d, d + N, d + 2 * N, d + 3 * N};
  for (int k = 0; k < 4; ++k) {
    if (!src[k]) continue;
    CK(c, cudaMemcpyAsync(dst[k], src[k], (k == 3 ? 2 : 1) * N * sizeof(double),
                          cudaMemcpyHostToDevice, c->stream));
  }
  void* uwx = u_wall ? c->wall_uwx : nullptr;
  void* uwy = u_wall ? c->wall_uwy : nullptr;
  cudaError_t e;
  if (c->p.storage == LBM_FP64) {
    auto f = c->Q == 9 ? launch_wall_prepare<9, double> : launch_wall_prepare<21, double>;
    e = f(phi_s ? dst[0] : nullptr, psi_r ? dst[1] : nullptr, psi_a ? dst[2] : nullptr,
          u_wall ? dst[3] : nullptr, G_R, G_A, epsilon, nx, ny, (double*)c->wall_phie,
          (double*)c->wall_sx, (double*)c->wall_sy, (double*)uwx, (double*)uwy, c->wall_flags,
          c->nchunk_pad, c->stream);
  } else {
    auto f = c->Q == 9 ? launch_wall_prepare<9, float> : launch_wall_prepare<21, float>;
    e = f(phi_s ? dst[0] : nullptr, psi_r ? dst[1] : nullptr, psi_a ? dst[2] : nullptr,
          u_wall ? dst[3] : nullptr, G_R, G_A, epsilon, nx, ny, (float*)c->wall_phie,
          (float*)c->wall_sx, (float*)c->wall_sy, (float*)uwx, (float*)uwy, c->wall_flags,
          c->nchunk_pad, c->stream);
  }
  CK(c, e);
  if (!u_wall && c->wall_uwx) {
    // keep the buffers but stop using them
    dfree(c, c->wall_uwx);
    dfree(c, c->wall_uwy);
    c->wall_uwx = c->wall_uwy = nullptr;
  }
  c->has_wall = phi_s || psi_r || psi_a;
  c->version += 1;
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
  int rc = guard(c);
  if (rc) return rc;
  if (!f) return fail(c, LBM_EINVAL, "null populations");
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  Tmp stage(c, (size_t)N * (c->Q + 1) * sizeof(double));
  if (!stage.p) return fail(c, LBM_ENOMEM, "population staging");
  double* d = stage.as<double>();
  CK(c, cudaMemcpyAsync(d, f, (size_t)N * c->Q * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(c, launch_colsum(d, c->Q, N, d + (int64_t)c->Q * N, c->stream));
  rc = set_shift_from_rho(c, d + (int64_t)c->Q * N);
  if (rc) return rc;
  rc = dispatch(c->Q, c->p.storage, [&]<int Q, typename S>() -> int {
    CK(c, launch_encode<Q, S>(d, static_cast<S*>(c->buf[c->cur]), c->p.nx, c->p.ny, c->pitch,
                              c->plane, c->rho_s, c->stream));
    return LBM_OK;
  });
  if (rc) return rc;
  CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream));
  CK(c, cudaMemsetAsync(c->d_status + kRngWord, 0, 2 * sizeof(uint32_t), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps = 0;
  c->version += 1;  // the shift (step arguments) may have changed
  return LBM_OK;
}

int lbm_set_equilibrium(lbm_ctx* c, const double* rho, const double* ux, const double* uy,
                        const double* dfi) {
  int rc = guard(c);
  if (rc) return rc;
  if (!rho || !ux || !uy) return fail(c, LBM_EINVAL, "null rho/ux/uy");
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  const int64_t extra = dfi ? (int64_t)c->Q * N : 0;
  Tmp stage(c, (size_t)(3 * N + extra) * sizeof(double));
  if (!stage.p) return fail(c, LBM_ENOMEM, "equilibrium staging");
  double* d = stage.as<double>();
  CK(c, cudaMemcpyAsync(d, rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(d + N, ux, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(d + 2 * N, uy, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (dfi)
    CK(c, cudaMemcpyAsync(d + 3 * N, dfi, extra * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  rc = set_shift_from_rho(c, d);
  if (rc) return rc;
  rc = dispatch(c->Q, c->p.storage, [&]<int Q, typename S>() -> int {
    CK(c, launch_equilibrium<Q, S>(d, d + N, d + 2 * N, dfi ? d + 3 * N : nullptr,
                                   static_cast<S*>(c->buf[c->cur]), c->p.nx, c->p.ny, c->pitch,
                                   c->plane, c->rho_s, c->stream));
    return LBM_OK;
  });
  if (rc) return rc;
  CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), c->stream));
  CK(c, cudaMemsetAsync(c->d_status + kRngWord, 0, 2 * sizeof(uint32_t), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->has_state = true;
  c->steps = 0;
  c->version += 1;  // the shift (step arguments) may have changed
  return LBM_OK;
}

static int read_status(lbm_ctx* c) {
  uint32_t h = 0;
  CK(c, cudaMemcpyAsync(&h, c->d_status, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (h & kStatusTimeout)
    return fail(c, LBM_ETIMEOUT, "a TMA stage wait timed out in the step kernel");
  if (h & kStatusNonFinite)
    return fail(c, LBM_ENONFINITE, "non-finite density after %lld steps", (long long)c->steps);
  return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t nsteps) {
  int rc = guard(c);
  if (rc) return rc;
  if (nsteps < 0) return fail(c, LBM_EINVAL, "negative step count");
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  for (int64_t s = 0; s < nsteps; ++s) {
    rc = dispatch(c->Q, c->p.storage, [&]<int Q, typename S>() -> int {
      return run_pass<Q, S>(c, kModeStep, nullptr, nullptr, nullptr, 0,
                            static_cast<S*>(c->buf[c->cur ^ 1]));
    });
    if (rc) return rc;
    c->stall_wait_ns = 0;  // the test hook covers one step
    c->cur ^= 1;
    c->steps += 1;
    if (c->p.check_every > 0 && c->steps % c->p.check_every == 0) {
      rc = read_status(c);
      if (rc) return rc;
    }
  }
  return LBM_OK;
}

int lbm_moments_device(lbm_ctx* c, double* d_rho, double* d_ux, double* d_uy) {
  int rc = guard(c);
  if (rc) return rc;
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  // The read-out pass writes all three arrays; route unwanted ones to scratch.
  Tmp scratch(c, (!d_rho || !d_ux || !d_uy) ? (size_t)N * sizeof(double) : 0);
  double* sink = scratch.as<double>();
  if ((!d_rho || !d_ux || !d_uy) && !sink) return fail(c, LBM_ENOMEM, "moments scratch");
  return dispatch(c->Q, c->p.storage, [&]<int Q, typename S>() -> int {
    return run_pass<Q, S>(c, kModeMoments, d_rho ? d_rho : sink, d_ux ? d_ux : sink,
                          d_uy ? d_uy : sink, 0, nullptr);
  });
}

int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy) {
  int rc = guard(c);
  if (rc) return rc;
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  Tmp stage(c, (size_t)3 * N * sizeof(double));
  if (!stage.p) return fail(c, LBM_ENOMEM, "moments staging");
  double* d = stage.as<double>();
  rc = lbm_moments_device(c, d, d + N, d + 2 * N);
  if (rc) return rc;
  double* hs[3] = {rho, ux, uy};
  for (int k = 0; k < 3; ++k)
    if (hs[k])
      CK(c, cudaMemcpyAsync(hs[k], d + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* f) {
  int rc = guard(c);
  if (rc) return rc;
  if (!f) return fail(c, LBM_EINVAL, "null output");
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  Tmp stage(c, (size_t)N * c->Q * sizeof(double));
  if (!stage.p) return fail(c, LBM_ENOMEM, "population staging");
  double* d = stage.as<double>();
  rc = dispatch(c->Q, c->p.storage, [&]<int Q, typename S>() -> int {
    CK(c, launch_decode<Q, S>(static_cast<const S*>(c->buf[c->cur]), d, c->p.nx, c->p.ny,
                              c->pitch, c->plane, c->rho_s, c->stream));
    return LBM_OK;
  });
  if (rc) return rc;
  CK(c, cudaMemcpyAsync(f, d, (size_t)N * c->Q * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_totals(lbm_ctx* c, double out[3]) {
  int rc = guard(c);
  if (rc) return rc;
  if (!out) return fail(c, LBM_EINVAL, "null output");
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  const int64_t N = (int64_t)c->p.nx * c->p.ny;
  Tmp stage(c, (size_t)3 * N * sizeof(double));
  if (!stage.p) return fail(c, LBM_ENOMEM, "totals staging");
  double* d = stage.as<double>();
  rc = dispatch(c->Q, c->p.storage, [&]<int Q, typename S>() -> int {
    return run_pass<Q, S>(c, kModeMoments, d, d + N, d + 2 * N, 1, nullptr);
  });
  if (rc) return rc;
  CK(c, launch_reduce3(d, d + N, d + 2 * N, N, c->d_partials, c->nparts, c->d_out3, c->stream));
  CK(c, cudaMemcpyAsync(out, c->d_out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int lbm_steps_done(const lbm_ctx* c, int64_t* out) {
  if (!c || !out) return fail(nullptr, LBM_EINVAL, "null argument");
  *out = c->steps;
  return LBM_OK;
}

int lbm_get_clock(lbm_ctx* c, int64_t* steps, uint32_t* rounding_counter, double* rho_s) {
  int rc = guard(c);
  if (rc) return rc;
  if (!steps || !rounding_counter) return fail(c, LBM_EINVAL, "null output");
  if (rho_s) *rho_s = c->rho_s;
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  uint32_t h = 0;
  CK(c, cudaMemcpyAsync(&h, c->d_status + kRngWord + c->cur, sizeof h, cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  *steps = c->steps;
  *rounding_counter = h;
  return LBM_OK;
}

int lbm_set_clock(lbm_ctx* c, int64_t steps, uint32_t rounding_counter) {
  int rc = guard(c);
  if (rc) return rc;
  if (steps < 0) return fail(c, LBM_EINVAL, "negative step count");
  if (!c->has_state) return fail(c, LBM_ESTATE, "populations not set");
  // The next step reads the counter word of the current buffer (see make_args).
  const uint32_t v = rounding_counter;
  CK(c, cudaMemcpyAsync(c->d_status + kRngWord + c->cur, &v, sizeof v, cudaMemcpyHostToDevice,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->steps = steps;
  return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
  int rc = guard(c);
  if (rc) return rc;
  CK(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

int lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_OK;
  cudaStreamSynchronize(c->stream);
  cudaGetLastError();
  std::vector<void*> live = c->owned;
  for (void* p : live) dfree(c, p);
  delete c;
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

int lbm_debug_stall_next_step(lbm_ctx* c, int32_t wait_ms) {
  int rc = guard(c);
  if (rc) return rc;
  if (wait_ms < 1) return fail(c, LBM_EINVAL, "wait_ms must be >= 1");
  c->stall_wait_ns = (uint64_t)wait_ms * 1000000ull;
  return LBM_OK;
}

int lbm_get_layout(const lbm_ctx* c, lbm_layout* out) {
  if (!c || !out) return fail(nullptr, LBM_EINVAL, "null argument");
  out->bytes_per_node = 2LL * c->Q * c->esize;
  out->pitch = c->pitch;
  out->strip_width = c->W;
  out->tile_rows = c->tile_rows;
  out->grid_x = c->grid_x;
  out->grid_y = c->grid_y;
  out->stages = c->NS;
  out->ghost_x = c->GX;
  out->ghost_y = c->GY;
  out->device_bytes = 2LL * c->plane * c->Q * c->esize;
  return LBM_OK;
}

int lbm_wall_gaussian_filter(int32_t nx, int32_t ny, int32_t lattice, const uint8_t* solid,
                             int32_t n_rep, int32_t n_att, double* phi_s, double* psi_r,
                             double* psi_a) {
  if (nx < 1 || ny < 1 || !solid || n_rep < 0 || n_att < n_rep ||
      (lattice != LBM_D2Q9 && lattice != LBM_D2Q21))
    return fail(nullptr, LBM_EINVAL, "wall filter arguments");
  const int64_t N = (int64_t)nx * ny;
  double* g[2] = {nullptr, nullptr};
  double* keep = nullptr;
  uint8_t* dsolid = nullptr;
  auto cleanup = [&] {
    cudaFree(g[0]);
    cudaFree(g[1]);
    cudaFree(keep);
    cudaFree(dsolid);
  };
  if (cudaMalloc(&g[0], N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&g[1], N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&keep, N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dsolid, N) != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    return fail(nullptr, LBM_ENOMEM, "wall filter buffers");
  }
  std::vector<double> h0(N);
  for (int64_t n = 0; n < N; ++n) h0[n] = solid[n] ? 1.0 : 0.0;
  cudaError_t e = cudaMemcpy(g[0], h0.data(), N * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dsolid, solid, N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n_rep == 0) e = cudaMemcpy(keep, g[0], N * sizeof(double), cudaMemcpyDeviceToDevice);
  int cur = 0;
  for (int it = 1; it <= n_att && e == cudaSuccess; ++it) {
    e = launch_filter_pass(lattice, g[cur], g[cur ^ 1], dsolid, nx, ny, nullptr);
    cur ^= 1;
    if (e == cudaSuccess && it == n_rep)
      e = cudaMemcpy(keep, g[cur], N * sizeof(double), cudaMemcpyDeviceToDevice);
  }
  std::vector<double> ga(N), gr(N);
  if (e == cudaSuccess) e = cudaMemcpy(ga.data(), g[cur], N * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(gr.data(), keep, N * sizeof(double), cudaMemcpyDeviceToHost);
  cleanup();
  if (e != cudaSuccess) return fail(nullptr, LBM_ECUDA, "wall filter: %s", cudaGetErrorString(e));
  for (int64_t n = 0; n < N; ++n) {
    if (phi_s) phi_s[n] = ga[n];
    if (psi_r) psi_r[n] = gr[n];
    if (psi_a) psi_a[n] = ga[n] - gr[n];
  }
  return LBM_OK;
}

int lbm_wall_core_tail(int32_t nx, int32_t ny, const double* dist, const double* thickness,
                       double core_lambda, double core_cut, double tail_exp, double tail_cut,
                       double phi_cut, double* phi_s, double* psi_r, double* psi_a) {
  if (nx < 1 || ny < 1 || !dist || !thickness || !(core_lambda > 0.0))
    return fail(nullptr, LBM_EINVAL, "core/tail arguments");
  const double rc = std::exp(-core_cut / core_lambda);
  const double tc = std::pow(1.0 + tail_cut, -tail_exp);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const int64_t n = (int64_t)y * nx + x;
      const double d = dist[n], T = thickness[x];
      double ph = 0.5 * (1.0 - std::tanh((d - 0.5 * T) / (0.25 * T)));
      if (ph < phi_cut) ph = 0.0;
      if (phi_s) phi_s[n] = ph;
      if (psi_r) psi_r[n] = d < core_cut ? std::exp(-d / core_lambda) - rc : 0.0;
      if (psi_a) psi_a[n] = d < tail_cut ? std::pow(1.0 + d, -tail_exp) - tc : 0.0;
    }
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batches: many lattices of one (lattice, storage) kind advanced together
// ---------------------------------------------------------------------------
}  // extern "C"

// Steps per replay of the batch's long captured graph (even: the graph
// returns the buffers to the parity it started from).
constexpr int kLongSteps = 16;
static_assert(kLongSteps % 2 == 0, "a replay must end on the parity it started from");

struct lbm_batch {
  lbm_allocator alloc{};
  bool user_alloc = false;
  cudaStream_t stream = nullptr;
  std::vector<lbm_ctx*> members;
  std::vector<uint64_t> versions;
  std::vector<int> cur0;  // member cur at build time
  int Q = 0, storage = -1;
  int tile_rows = 0;  // 0: each member's own choice
  int ctas = 0;       // 0: one CTA per tile; > 0: that many persistent CTAs
  bool dirty = true;
  void* d_members = nullptr;
  size_t cap_members = 0;
  int ntiles = 0, nctas = 0;
  int64_t phase = 0;
  cudaGraphExec_t gexec = nullptr;       // two steps
  cudaGraphExec_t gexec_long = nullptr;  // kLongSteps steps
  cudaEvent_t order_ev = nullptr;  // orders member streams with the batch stream
  // Members are launched in chunks of up to BatchArgs::kChunk, each with its step
  // arguments as a kernel parameter.  With several chunks every chunk has its
  // own stream, forked from and joined back to the batch stream around each
  // sequence of steps (a member depends only on its own previous step).
  struct Chunk {
    std::vector<unsigned char> args;  // host copy of BatchArgs<T, S>
    int base = 0, count = 0;          // members [base, base + count)
    int nctas = 0;
    bool plain = false;               // every member: exponential psi, no projection, SR
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Chunk> chunks;
  cudaEvent_t fork_ev = nullptr;
  std::string err;
  bool poisoned = false;
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (b) {
    b->err = msg;
    if (code == LBM_ECUDA) b->poisoned = true;
  } else {
    g_err = msg;
  }
  return code;
}

#define BCK(b, ...)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (__VA_ARGS__);                                                    \
    if (e_ != cudaSuccess)                                                             \
      return bfail((b), LBM_ECUDA, "%s failed: %s", #__VA_ARGS__, cudaGetErrorString(e_)); \
  } while (0)

void* balloc(lbm_batch* b, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (b->user_alloc)
    p = b->alloc.alloc(bytes, b->alloc.user);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void bfree(lbm_batch* b, void* p) {
  if (!p) return;
  if (b->user_alloc)
    b->alloc.free(p, b->alloc.user);
  else
    cudaFree(p);
}

int bgrow(lbm_batch* b, void** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return LBM_OK;
  if (*p) {
    cudaStreamSynchronize(b->stream);
    bfree(b, *p);
  }
  *p = balloc(b, need);
  *cap = *p ? need : 0;
  return *p ? LBM_OK : bfail(b, LBM_ENOMEM, "batch descriptor of %zu bytes", need);
}

void drop_graph(lbm_batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (b->gexec_long) {
    cudaGraphExecDestroy(b->gexec_long);
    b->gexec_long = nullptr;
  }
}

void release_chunk(lbm_batch::Chunk& ch) {
  if (ch.stream) {
    cudaStreamSynchronize(ch.stream);
    cudaStreamDestroy(ch.stream);
  }
  if (ch.done) cudaEventDestroy(ch.done);
  ch.stream = nullptr;
  ch.done = nullptr;
}

template <int Q, typename S> int batch_build(lbm_batch* b) {
  using T = typename Codec<S>::T;
  using M = BatchMember<T, S>;
  using A = BatchArgs<T, S>;
  constexpr int W = StepConfig<Q, S>::W;
  const int n = (int)b->members.size();
  constexpr int kChunk = A::kChunk;
  const int nchunk = (n + kChunk - 1) / kChunk;
  std::vector<M> hm(n);
  b->versions.assign(n, 0);
  b->cur0.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    lbm_ctx* c = b->members[i];
    M& m = hm[i];
    std::memset(&m, 0, sizeof m);
    m.map[0] = c->tmap[0];
    m.map[1] = c->tmap[1];
    m.flags = c->has_wall ? c->flag_map : c->tmap[0].m[0];
    b->versions[i] = c->version;
    b->cur0[i] = c->cur;
  }
  for (size_t k = nchunk; k < b->chunks.size(); ++k) release_chunk(b->chunks[k]);
  b->chunks.resize(nchunk);
  // Tiles per chunk, member by member; within a member segment by segment
  // (all strips of a segment before the next).  The kernel derives each
  // CTA's tile from its block index and these counts.
  size_t total = 0;
  std::vector<int> chunk_tiles(nchunk, 0);
  for (int k = 0; k < nchunk; ++k) {
    lbm_batch::Chunk& ch = b->chunks[k];
    ch.base = k * kChunk;
    ch.count = std::min(kChunk, n - ch.base);
    ch.args.assign(sizeof(A), 0);
    A* pa = reinterpret_cast<A*>(ch.args.data());
    ch.plain = true;
    int32_t t0 = 0;
    for (int i = 0; i < ch.count; ++i) {
      lbm_ctx* c = b->members[ch.base + i];
      ch.plain = ch.plain && c->p.psi_kind == LBM_PSI_EXP && !c->p.project &&
                 (!Codec<S>::kShifted || c->p.rounding == LBM_ROUND_STOCHASTIC);
      for (int d = 0; d < 2; ++d)
        pa->a[i][d] = make_args<Q, S>(c, d, static_cast<S*>(c->buf[d ^ 1]), nullptr, nullptr, nullptr, 0);
      pa->cur[i] = c->cur;
      // Segments of about L rows, balanced over the member's height: a short
      // remainder segment would pay its 2R halo rows and its pipeline fill
      // for a few rows only.
      const int L = std::max(1, std::min(b->tile_rows > 0 ? b->tile_rows : c->tile_rows, c->p.ny));
      pa->nseg[i] = std::max(1, (c->p.ny + L / 2) / L);
      pa->nstrip[i] = (c->p.nx + W - 1) / W;
      pa->tile0[i] = t0;
      t0 += pa->nseg[i] * pa->nstrip[i];
    }
    for (int i = ch.count; i <= kChunk; ++i) pa->tile0[i] = t0;
    chunk_tiles[k] = t0;
    total += (size_t)t0;
  }
  b->nctas = 0;
  for (int k = 0; k < nchunk; ++k) {
    lbm_batch::Chunk& ch = b->chunks[k];
    // Persistent CTAs: the batch's count shared out by tiles; CTA j of a
    // chunk marches its tiles j, j + G, ...
    ch.nctas = b->ctas <= 0
                   ? chunk_tiles[k]
                   : (int)std::max<int64_t>(
                         1, std::min<int64_t>(chunk_tiles[k],
                                              std::llround((double)b->ctas * chunk_tiles[k] / total)));
    b->nctas += ch.nctas;
    if (nchunk > 1 && !ch.stream) {
      BCK(b, cudaStreamCreateWithFlags(&ch.stream, cudaStreamNonBlocking));
      BCK(b, cudaEventCreateWithFlags(&ch.done, cudaEventDisableTiming));
    }
  }
  if (nchunk > 1 && !b->fork_ev) BCK(b, cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
  b->ntiles = (int)total;
  batch_ctas_per_sm<Q, S>();  // sets the kernel's shared-memory attribute outside any capture
  int rc = bgrow(b, &b->d_members, &b->cap_members, sizeof(M) * std::max(1, n));
  if (rc) return rc;
  BCK(b, cudaMemcpyAsync(b->d_members, hm.data(), sizeof(M) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));  // host vectors go out of scope
  b->phase = 0;
  drop_graph(b);
  b->dirty = false;
  return LBM_OK;
}

// Enqueues one step of every chunk (on its own stream when there are several;
// the caller forks and joins them).
template <int Q, typename S> cudaError_t batch_launch(lbm_batch* b, int parity) {
  using T = typename Codec<S>::T;
  const bool multi = b->chunks.size() > 1;
  for (const lbm_batch::Chunk& ch : b->chunks) {
    cudaError_t e = launch_batch<Q, S>(
        *reinterpret_cast<const BatchArgs<T, S>*>(ch.args.data()),
        static_cast<const BatchMember<T, S>*>(b->d_members) + ch.base, ch.nctas, parity,
        b->ctas > 0, ch.plain, multi ? ch.stream : b->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int batch_guard(lbm_batch* b) {
  if (!b) return bfail(nullptr, LBM_EINVAL, "null batch");
  if (b->poisoned) return bfail(b, LBM_ESTATE, "batch poisoned by an earlier CUDA error: %s", b->err.c_str());
  return LBM_OK;
}

// Rebuilds the descriptors when a member changed (walls, stream) or was
// stepped on its own since the last build.
int batch_refresh(lbm_batch* b) {
  if (!b->dirty) {
    for (size_t i = 0; i < b->members.size(); ++i) {
      const lbm_ctx* c = b->members[i];
      if (c->version != b->versions[i] || c->cur != (b->cur0[i] ^ (int)(b->phase & 1))) {
        b->dirty = true;
        break;
      }
    }
  }
  if (!b->dirty) return LBM_OK;
  for (lbm_ctx* c : b->members) {
    if (c->poisoned) return bfail(b, LBM_ESTATE, "a member context is poisoned");
    if (!c->has_state) return bfail(b, LBM_ESTATE, "a member has no populations");
  }
  return dispatch(b->Q, b->storage, [&]<int Q, typename S>() { return batch_build<Q, S>(b); });
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_allocator* a, void* cuda_stream, lbm_batch** out) {
  if (!out) return bfail(nullptr, LBM_EINVAL, "null output pointer");
  *out = nullptr;
  if (a && (!a->alloc || !a->free)) return bfail(nullptr, LBM_EINVAL, "allocator without alloc/free");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation");
  if (a) {
    b->alloc = *a;
    b->user_alloc = true;
  }
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = b;
  return LBM_OK;
}

int lbm_batch_add(lbm_batch* b, lbm_ctx* c) {
  int rc = batch_guard(b);
  if (rc) return rc;
  if (!c) return bfail(b, LBM_EINVAL, "null member");
  if (std::find(b->members.begin(), b->members.end(), c) != b->members.end())
    return bfail(b, LBM_EINVAL, "context already in the batch");
  if (!b->members.empty() && (c->Q != b->Q || c->p.storage != b->storage))
    return bfail(b, LBM_EINVAL, "members must share lattice and storage (batch: D2Q%d/%d, member: D2Q%d/%d)",
                 b->Q, b->storage, c->Q, c->p.storage);
  if (b->members.empty()) {
    b->Q = c->Q;
    b->storage = c->p.storage;
  }
  b->members.push_back(c);
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_remove(lbm_batch* b, lbm_ctx* c) {
  int rc = batch_guard(b);
  if (rc) return rc;
  auto it = std::find(b->members.begin(), b->members.end(), c);
  if (it == b->members.end()) return bfail(b, LBM_EINVAL, "context not in the batch");
  b->members.erase(it);
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_size(const lbm_batch* b, int32_t* n) {
  if (!b || !n) return bfail(nullptr, LBM_EINVAL, "null argument");
  *n = (int32_t)b->members.size();
  return LBM_OK;
}

int lbm_batch_launches_per_step(const lbm_batch* b, int32_t* n) {
  if (!b || !n) return bfail(nullptr, LBM_EINVAL, "null argument");
  const int chunk = b->storage == LBM_FP64 ? batch_chunk<double>() : batch_chunk<float>();
  *n = (int32_t)((b->members.size() + chunk - 1) / chunk);
  return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch* b, int32_t tile_rows, int32_t ctas) {
  int rc = batch_guard(b);
  if (rc) return rc;
  if (tile_rows < 0 || ctas < 0) return bfail(b, LBM_EINVAL, "negative tiling");
  b->tile_rows = tile_rows;
  b->ctas = ctas;
  b->dirty = true;
  return LBM_OK;
}

namespace {
// Tilings chosen by lbm_batch_autotune, per (lattice, storage, size class):
// the size class is floor(log2(nodes)) of the batch's total node count and
// floor(log2(members)).  Process-wide, shared by every batch.
struct TuneKey {
  int q, storage, nodes_log2, members_log2;
  bool operator<(const TuneKey& o) const {
    return std::tie(q, storage, nodes_log2, members_log2) <
           std::tie(o.q, o.storage, o.nodes_log2, o.members_log2);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tuned;

int floor_log2(int64_t v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

TuneKey tune_key(const lbm_batch* b) {
  int64_t nodes = 0;
  for (const lbm_ctx* c : b->members) nodes += (int64_t)c->p.nx * c->p.ny;
  return TuneKey{b->Q, b->storage, floor_log2(nodes), floor_log2((int64_t)b->members.size())};
}
}  // namespace

int lbm_batch_use_tuned(lbm_batch* b, int32_t* found) {
  int rc = batch_guard(b);
  if (rc) return rc;
  if (!found) return bfail(b, LBM_EINVAL, "null argument");
  *found = 0;
  if (b->members.empty()) return LBM_OK;
  std::pair<int, int> t;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(tune_key(b));
    if (it == g_tuned.end()) return LBM_OK;
    t = it->second;
  }
  if (t.first != b->tile_rows || t.second != b->ctas) {
    b->tile_rows = t.first;
    b->ctas = t.second;
    b->dirty = true;
  }
  *found = 1;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
  int rc = batch_guard(b);
  if (rc) return rc;
  if (nsteps < 0) return bfail(b, LBM_EINVAL, "negative step count");
  if (b->members.empty() || nsteps == 0) return LBM_OK;
  rc = batch_refresh(b);
  if (rc) return rc;
  // Work already enqueued on the members' own streams (initialisation,
  // read-outs) completes before the batch touches their buffers.
  if (!b->order_ev) BCK(b, cudaEventCreateWithFlags(&b->order_ev, cudaEventDisableTiming));
  std::vector<cudaStream_t> mstreams;
  for (lbm_ctx* c : b->members)
    if (c->stream != b->stream &&
        std::find(mstreams.begin(), mstreams.end(), c->stream) == mstreams.end())
      mstreams.push_back(c->stream);
  for (cudaStream_t ms : mstreams) {
    BCK(b, cudaEventRecord(b->order_ev, ms));
    BCK(b, cudaStreamWaitEvent(b->stream, b->order_ev, 0));
  }
  // Steps with the given parities: fork the chunk streams from the batch
  // stream, launch each chunk's steps on its stream, join them back.
  // Steps with parities parity0, parity0 ^ 1, ... (n of them).
  auto launch = [&](int parity0, int n) -> int {
    const bool multi = b->chunks.size() > 1;
    if (multi) {
      BCK(b, cudaEventRecord(b->fork_ev, b->stream));
      for (const lbm_batch::Chunk& ch : b->chunks) BCK(b, cudaStreamWaitEvent(ch.stream, b->fork_ev, 0));
    }
    for (int j = 0; j < n; ++j) {
      const int parity = parity0 ^ (j & 1);
      const int r = dispatch(b->Q, b->storage, [&]<int Q, typename S>() -> int {
        BCK(b, batch_launch<Q, S>(b, parity));
        return LBM_OK;
      });
      if (r) return r;
    }
    if (multi) {
      for (const lbm_batch::Chunk& ch : b->chunks) {
        BCK(b, cudaEventRecord(ch.done, ch.stream));
        BCK(b, cudaStreamWaitEvent(b->stream, ch.done, 0));
      }
    }
    return LBM_OK;
  };
  int64_t left = nsteps;
  // Bring the phase to even, then replay captured graphs of kLongSteps steps
  // (the chunk streams join once per graph) and of two steps.
  if (b->phase & 1) {
    if ((rc = launch(1, 1))) return rc;
    b->phase += 1;
    left -= 1;
  }
  auto capture = [&](int n, cudaGraphExec_t* out) -> int {
    cudaGraph_t graph = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    const int r = launch(0, n);
    cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
    if (r) {
      if (graph) cudaGraphDestroy(graph);
      return r;
    }
    BCK(b, ee);
    cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    BCK(b, ei);
    return LBM_OK;
  };
  if (left >= kLongSteps && b->stream != nullptr && !b->gexec_long) {
    if ((rc = capture(kLongSteps, &b->gexec_long))) return rc;
  }
  while (left >= kLongSteps && b->gexec_long) {
    BCK(b, cudaGraphLaunch(b->gexec_long, b->stream));
    b->phase += kLongSteps;
    left -= kLongSteps;
  }
  if (left >= 2 && b->stream != nullptr && !b->gexec) {
    if ((rc = capture(2, &b->gexec))) return rc;
  }
  while (left >= 2) {
    if (b->gexec) {
      BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    } else {
      if ((rc = launch(0, 2))) return rc;
    }
    b->phase += 2;
    left -= 2;
  }
  if (left == 1) {
    if ((rc = launch(0, 1))) return rc;
    b->phase += 1;
  }
  // Later work on a member's stream sees the batch's steps.
  BCK(b, cudaEventRecord(b->order_ev, b->stream));
  for (cudaStream_t ms : mstreams) BCK(b, cudaStreamWaitEvent(ms, b->order_ev, 0));
  for (lbm_ctx* c : b->members) {
    c->cur ^= (int)(nsteps & 1);
    c->steps += nsteps;
  }
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int32_t steps_per_trial, int32_t* best_tile_rows,
                       int32_t* best_ctas, double* best_ms_per_step) {
  int rc = batch_guard(b);
  if (rc) return rc;
  if (b->members.empty() || steps_per_trial < 1) return bfail(b, LBM_EINVAL, "empty batch or no steps");
  int dev = 0, sms = 0;
  BCK(b, cudaGetDevice(&dev));
  BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int cps = dispatch(b->Q, b->storage, [&]<int Q, typename S>() { return batch_ctas_per_sm<Q, S>(); });
  const int rows_c[] = {4, 8, 12, 16, 24, 32, 64};
  const int ctas_c[] = {0, std::max(1, cps) * sms};
  cudaEvent_t e0, e1;
  BCK(b, cudaEventCreate(&e0));
  BCK(b, cudaEventCreate(&e1));
  double best = 1e300;
  int bt = b->tile_rows, bc = b->ctas;
  for (int tr : rows_c) {
    for (int ct : ctas_c) {
      b->tile_rows = tr;
      b->ctas = ct;
      b->dirty = true;
      // warm-up: rebuild, capture both graphs
      if ((rc = lbm_batch_step(b, kLongSteps + 2))) break;
      cudaEventRecord(e0, b->stream);
      if ((rc = lbm_batch_step(b, steps_per_trial))) break;
      cudaEventRecord(e1, b->stream);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = bfail(b, LBM_ECUDA, "autotune timing failed");
        break;
      }
      const double per = ms / steps_per_trial;
      if (per < best) {
        best = per;
        bt = tr;
        bc = ct;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->tile_rows = bt;
  b->ctas = bc;
  b->dirty = true;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[tune_key(b)] = {bt, bc};
  }
  if (best_tile_rows) *best_tile_rows = bt;
  if (best_ctas) *best_ctas = bc;
  if (best_ms_per_step) *best_ms_per_step = best;
  return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  cudaStreamSynchronize(b->stream);
  cudaGetLastError();
  drop_graph(b);
  for (lbm_batch::Chunk& ch : b->chunks) release_chunk(ch);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->order_ev) cudaEventDestroy(b->order_ev);
  bfree(b, b->d_members);
  delete b;
  return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_err.c_str(); }

}  // extern "C"

