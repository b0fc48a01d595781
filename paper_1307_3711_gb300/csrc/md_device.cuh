// md_device.cuh -- device code of the laser-cluster MD hot path for sm_103a.
//
// Method (Holkundkar, arXiv:1307.3711, Sec. II): every particle moves under the
// Coulomb field of all other charged particles plus the spatially uniform laser
// field of Eqs. 3-9 (b0 = a0), advanced by a relativistic Boris leap-frog.
//
// Design for GB300 (not the paper's OpenMP decomposition):
//   * the j-stream is an SoA float4 array (x, y, z, K_C*Q) double-buffered
//     across steps; tiles of it are staged into shared memory by 1-D TMA bulk
//     copies (cp.async.bulk) completing on an mbarrier, STAGES deep;
//   * each thread keeps R i-particles in registers (register blocking), every
//     source is one broadcast LDS.128 shared by R pair evaluations;
//   * one pair is 12 FP32-pipe instructions (3 FADD, 3 FFMA, 3 FMUL, 3 FFMA)
//     plus one MUFU.RSQ (rsqrt.approx.ftz.f32);
//   * FP32 partial sums are folded into Kahan-compensated FP32 sums once per
//     tile, so the compensation costs ~12/TILE instructions per pair;
//   * the laser field and the Boris kick are fused into the epilogue: the
//     kick increment is evaluated in FP32, the integrator state (x, u) and the
//     drift are FP64;
//   * shares of work units (cluster, i-block, piece of the sources) are
//     handed out by an atomic ticket to a persistent grid, so uneven clusters
//     of a parameter scan share one launch; the last CTA to finish resets the
//     ticket and advances the step counter, so a captured CUDA graph of many
//     steps replays without host work.
// Every mbarrier wait is bounded by a clock64 budget; on expiry the kernel sets
// an error bit, drains its own copies (again bounded) and returns.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "md_types.cuh"

namespace md {

// ------------------------------------------------------------------ PTX --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D TMA bulk copy global -> shared, completion counted on `bar` in bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`: false after `budget` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long budget = kWaitBudget) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Bounds checks of the checked build (-DMD_CHECKED): an index outside
// [lo, hi) sets kErrBounds in the error word and the access is skipped; the
// normal build compiles them away.
__device__ __forceinline__ bool in_range_checked(int* err, long long v, long long lo,
                                                 long long hi) {
  if (v >= lo && v < hi) return true;
  atomicOr(err, kErrBounds);
  return false;
}
#ifdef MD_CHECKED
#define MD_IN_RANGE(err, v, lo, hi) ::md::in_range_checked((err), (v), (lo), (hi))
#else
#define MD_IN_RANGE(err, v, lo, hi) true
#endif

// Explicit shared-memory loads (the tiles are reached through references, so
// the address space is stated rather than inferred).
__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr));
  return v;
}

__device__ __forceinline__ float lds_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ ulonglong2 lds_u64x2(uint32_t addr) {
  ulonglong2 v;
  asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(addr));
  return v;
}

__device__ __forceinline__ float rsqrt_mufu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------------- Philox ----
// Philox4x32-10 block function (Salmon et al., SC'11): per round, the 32x32
// products of words 0 and 2 with 0xD2511F53 / 0xCD9E8D57, high halves mixed
// with words 1 / 3 and the key; the key advances by 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    if (r < 9) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
  }
  return c;
}

// ------------------------------------------------- ionization rates (FP64) --
// Static ADK tunnelling and Lotz electron-impact rates of Sec. II's ionization
// paragraph, shared by the ionization pass and the surrogate's training data.

namespace rate {
constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;
constexpr double kHartreeEv = 27.211386245988;
constexpr double kFieldAu = 5.14220674763e11;   // V/m
constexpr double kTimeAu = 2.4188843265857e-17;  // s
constexpr double kMeC2Ev = 510998.95;
constexpr double kElemCharge = 1.602176634e-19;  // C
constexpr double kElectronMass = 9.1093837015e-31;  // kg
constexpr double kLotzA = 4.5e-14;               // cm^2 eV^2

// ---------------------------------------------------------------- rates ---

// E1(x) = int_x^inf e^-t/t dt: power series up to 1, even continued fraction
// (modified Lentz) beyond.
__device__ inline double expint_e1(double x) {
  if (!(x > 0.0)) return __longlong_as_double(0x7ff0000000000000LL);  // +inf
  if (x <= 1.0) {
    double sum = 0.0, term = 1.0;
    for (int k = 1; k < 60; ++k) {
      term *= -x / k;
      const double add = -term / k;
      sum += add;
      if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return -kEulerGamma - log(x) + sum;
  }
  const double tiny = 1e-300;
  double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 300; ++i) {
    const double an = -static_cast<double>(i) * i;
    b += 2.0;
    d = 1.0 / (an * d + b);
    c = b + an / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

// Static ADK rate (a.u.) at field F (a.u.), potential ip (a.u.), residual
// charge Z: n* = Z/sqrt(2 ip), l* = n* - 1, l = m = 0.
__device__ inline double adk_rate_au(double F, double ip, double Z) {
  if (!(F > 0.0)) return 0.0;
  const double ns = Z / sqrt(2.0 * ip);
  const double ls = ns - 1.0;
  const double c2 = pow(2.0, 2.0 * ns) / (ns * tgamma(ns + ls + 1.0) * tgamma(ns - ls));
  const double f0 = pow(2.0 * ip, 1.5);
  return c2 * ip * pow(2.0 * f0 / F, 2.0 * ns - 1.0) * exp(-2.0 * f0 / (3.0 * F));
}

// Lotz rate coefficient (cm^3/s): sqrt(8/(pi m_e)) a q E1(P/T) / (P sqrt(T)).
__device__ inline double lotz_rate_cgs(double P, double T, double q) {
  if (!(T > 0.0) || !(q > 0.0)) return 0.0;
  const double v_th = sqrt(8.0 * kElemCharge / (kPi * kElectronMass)) * 100.0;
  return v_th * kLotzA * q * expint_e1(P / T) / (P * sqrt(T));
}

// Total rate per unit time 1/omega of charge state z at |a| (paper units),
// ne (cm^-3), te (eV).
__device__ inline double rate_plain(const IonDev& io, double a_mag, int z, double ne, double te) {
  const double F = a_mag * kMeC2Ev * io.k_si / kFieldAu;
  const double w_ofi = adk_rate_au(F, io.ip_ev[z] / kHartreeEv, static_cast<double>(z + 1)) /
                       kTimeAu;
  const double w_ci = ne > 0.0 ? ne * lotz_rate_cgs(io.ip_ev[z], te, io.q_outer[z]) : 0.0;
  return (w_ofi + w_ci) / io.omega;
}

}  // namespace rate

// --------------------------------------------------------------- laser --

// Field-amplitude envelope (Eq. 3 and its readings): 0 Gaussian with
// intensity FWHM tau peaking at 2 tau; 1 sin^2(pi t/tau) on [0, tau];
// 2 exp[-2.77 (t-2tau)^2/tau^2] as printed; 3 flat.
__device__ __forceinline__ double envelope(double t, int kind, double tau) {
  if (kind == 0) {
    const double s = (t - 2.0 * tau) / tau;
    return exp(-1.3862943611198906 * s * s);  // 2 ln 2
  }
  if (kind == 1) {
    if (t < 0.0 || t > tau) return 0.0;
    const double s = sinpi(t / tau);
    return s * s;
  }
  if (kind == 2) {
    const double s = (t - 2.0 * tau) / tau;
    return exp(-2.77 * s * s);
  }
  return 1.0;
}

// Eqs. 4-9 at time t: linear E = A sin t x, B = A sin t y; circular adds
// E_y = A sin(t + 3pi/2) = -A cos t and B_x = A sin(t + pi/2) = A cos t.
// out = (a_x, a_y, a_z, b_x, b_y, b_z).
__device__ __forceinline__ void laser_field(const ClusterDev& c, double t, float* out) {
  const double amp = c.a0 * envelope(t, c.env, c.tau);
  double sn, cs;
  sincos(t, &sn, &cs);
  const double circ = c.pol ? 1.0 : 0.0;
  out[0] = static_cast<float>(amp * sn);
  out[1] = static_cast<float>(-circ * amp * cs);
  out[2] = 0.0f;
  out[3] = static_cast<float>(circ * amp * cs);
  out[4] = static_cast<float>(amp * sn);
  out[5] = 0.0f;
}

// ---------------------------------------------------------------- Boris --

// Increment du = u^{n+1/2} - u^{n-1/2} of one relativistic Boris kick
// (half electric kick, rotation with tan(theta/2) = h|b|/gamma, half
// electric kick), h = (q/m) dt / 2, evaluated in FP32.
__device__ __forceinline__ void boris_increment(float ux, float uy, float uz, float ex, float ey,
                                                float ez, float bx, float by, float bz, float h,
                                                float& dux, float& duy, float& duz) {
  const float hex = h * ex, hey = h * ey, hez = h * ez;
  const float mx = ux + hex, my = uy + hey, mz = uz + hez;
  const float ginv = rsqrtf(1.0f + mx * mx + my * my + mz * mz);
  const float tx = h * bx * ginv, ty = h * by * ginv, tz = h * bz * ginv;
  const float f = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
  const float sx = f * tx, sy = f * ty, sz = f * tz;
  const float px = mx + (my * tz - mz * ty);
  const float py = my + (mz * tx - mx * tz);
  const float pz = mz + (mx * ty - my * tx);
  // u+ - u- = u' x s ; total increment = 2 h E + u' x s
  dux = 2.0f * hex + (py * sz - pz * sy);
  duy = 2.0f * hey + (pz * sx - px * sz);
  duz = 2.0f * hez + (px * sy - py * sx);
}

__device__ __forceinline__ double wrap_periodic(double v, double box) {
  return v - box * floor((v + 0.5 * box) / box);
}

// ------------------------------------------------------- pair kernel body --

template <int R, bool POT>
struct Acc {
  float ax[R], ay[R], az[R], ap[R];  // FP32 partial over the current tile
  float sx[R], sy[R], sz[R], sp[R];  // Kahan sums
  float cx[R], cy[R], cz[R], cp[R];  // Kahan compensations

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ax[r] = ay[r] = az[r] = ap[r] = 0.0f;
      sx[r] = sy[r] = sz[r] = sp[r] = 0.0f;
      cx[r] = cy[r] = cz[r] = cp[r] = 0.0f;
    }
  }
};

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Minimum-image reduction of one displacement component in a periodic cube
// of side L (invL = 1/L): d - L rint(d / L), rounded to nearest even on the
// FP32 pipe by adding and removing 1.5 * 2^23 (|d / L| < 2^22).
__device__ __forceinline__ float min_image(float d, float L, float invL) {
  const float k = __fsub_rn(__fmaf_rn(d, invL, 12582912.0f), 12582912.0f);
  return __fmaf_rn(-L, k, d);
}

// One source against R targets: acc += Q_j (x_j - x_i) / (r^2 + eps^2)^{3/2}
// (and phi += Q_j / sqrt(r^2 + eps^2)); Q_j already carries K_C.  MI: the
// displacement is the minimum image in the periodic cube of side L.
template <int R, bool POT, bool MI = false>
__device__ __forceinline__ void pair(const float4 p, const float (&xi)[R], const float (&yi)[R],
                                     const float (&zi)[R], float eps2, Acc<R, POT>& a,
                                     float L = 0.0f, float invL = 0.0f) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float dx = p.x - xi[r];
    float dy = p.y - yi[r];
    float dz = p.z - zi[r];
    if constexpr (MI) {
      dx = min_image(dx, L, invL);
      dy = min_image(dy, L, invL);
      dz = min_image(dz, L, invL);
    }
    float r2 = fmaf(dx, dx, eps2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    const float ri = rsqrt_mufu(r2);
    const float qr = p.w * ri;
    const float ri2 = ri * ri;
    const float s = qr * ri2;
    a.ax[r] = fmaf(dx, s, a.ax[r]);
    a.ay[r] = fmaf(dy, s, a.ay[r]);
    a.az[r] = fmaf(dz, s, a.az[r]);
    if (POT) a.ap[r] += qr;
  }
}

// The same for a tile whose sources all carry one charge Q: the sum of
// (x_j - x_i)/(r^2+eps^2)^{3/2} (and 1/sqrt(r^2+eps^2)) without Q, which then
// multiplies the tile partial once (fold_q).  One FP32 multiply less per pair.
template <int R, bool POT, bool MI = false>
__device__ __forceinline__ void pair_u(const float4 p, const float (&xi)[R], const float (&yi)[R],
                                       const float (&zi)[R], float eps2, Acc<R, POT>& a,
                                       float L = 0.0f, float invL = 0.0f) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float dx = p.x - xi[r];
    float dy = p.y - yi[r];
    float dz = p.z - zi[r];
    if constexpr (MI) {
      dx = min_image(dx, L, invL);
      dy = min_image(dy, L, invL);
      dz = min_image(dz, L, invL);
    }
    float r2 = fmaf(dx, dx, eps2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    const float ri = rsqrt_mufu(r2);
    const float ri2 = ri * ri;
    const float s = ri2 * ri;
    a.ax[r] = fmaf(dx, s, a.ax[r]);
    a.ay[r] = fmaf(dy, s, a.ay[r]);
    a.az[r] = fmaf(dz, s, a.az[r]);
    if (POT) a.ap[r] += ri;
  }
}

// Whether all cnt sources of a landed tile carry the charge of the first one
// (q receives it).  Each warp decides for itself from the same shared data.
__device__ __forceinline__ bool tile_uniform_q(uint32_t tile, int cnt, float& q) {
  q = lds_f32(tile + 12u);
  bool ok = true;
  for (int k = static_cast<int>(threadIdx.x & 31u); k < cnt; k += 32)
    ok = ok && (lds_f32(tile + 16u * k + 12u) == q);
  return __all_sync(0xffffffffu, ok);
}

template <int R, bool POT>
__device__ __forceinline__ void fold(Acc<R, POT>& a) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    kahan_add(a.sx[r], a.cx[r], a.ax[r]);
    kahan_add(a.sy[r], a.cy[r], a.ay[r]);
    kahan_add(a.sz[r], a.cz[r], a.az[r]);
    a.ax[r] = a.ay[r] = a.az[r] = 0.0f;
    if (POT) {
      kahan_add(a.sp[r], a.cp[r], a.ap[r]);
      a.ap[r] = 0.0f;
    }
  }
}

// The tile partial of a charge-uniform tile times its charge, then folded.
// The products are rounded on their own (__fmul_rn), not fused into the
// Kahan subtraction that follows, so the scalar and packed paths (whose
// packed multiply is never fused) give the same bits.
template <int R, bool POT>
__device__ __forceinline__ void fold_q(Acc<R, POT>& a, float q) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a.ax[r] = __fmul_rn(a.ax[r], q);
    a.ay[r] = __fmul_rn(a.ay[r], q);
    a.az[r] = __fmul_rn(a.az[r], q);
    if (POT) a.ap[r] = __fmul_rn(a.ap[r], q);
  }
  fold<R, POT>(a);
}

// Shared-memory staging of the j-stream.
template <int TILE, int STAGES>
struct Stage {
  alignas(128) float4 tile[STAGES][TILE];
  alignas(8) uint64_t full[STAGES];
};

template <int TILE, int STAGES>
__device__ __forceinline__ void issue_tile(Stage<TILE, STAGES>& sm, unsigned g, const float4* src,
                                           long long ns, int t) {
  const int s = static_cast<int>(g % STAGES);
  const long long j0 = static_cast<long long>(t) * TILE;
  const long long rem = ns - j0;
  const uint32_t cnt = static_cast<uint32_t>(rem < TILE ? rem : TILE);
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&sm.full[s], cnt * 16u);
  bulk_g2s(&sm.tile[s][0], src + j0, cnt * 16u, &sm.full[s]);
}

// Whether any record in [r0, r1] lies in a live group (no flags: all live).
__device__ __forceinline__ bool any_live(const unsigned char* live, long long r0, long long r1) {
  if (!live) return true;
  for (long long g = r0 / kLiveGroup; g <= r1 / kLiveGroup; ++g)
    if (live[g]) return true;
  return false;
}

// First tile index >= t of a source range (ns records from global record
// gbase, tiles of `tile` records) that overlaps a live group, or ntiles if
// none does (no flags: t itself).  Dead tiles are neither copied nor summed.
__device__ __forceinline__ int next_live_tile(const unsigned char* live, long long gbase,
                                              long long ns, int t, int ntiles, int tile) {
  if (!live || t >= ntiles) return t;
  const long long r = gbase + static_cast<long long>(t) * tile;
  const long long gend = (gbase + ns - 1) / kLiveGroup;
  long long g = r / kLiveGroup;
  while (g <= gend && !live[g]) ++g;
  if (g > gend) return ntiles;
  const long long rr = g * kLiveGroup > r ? g * kLiveGroup : r;
  return static_cast<int>((rr - gbase) / tile);
}

// Sum over all ns sources for the R targets held by this thread, streaming the
// sources through the STAGES-deep TMA ring.  `it` counts tiles this CTA has
// consumed so far (sets the barrier phases).  Returns false (uniformly across
// the CTA) if a wait ran out of budget; the error bit is then set and this
// CTA's copies in flight have been waited for (bounded).
// Bounds of a landed tile's positions (same answer in every warp).
__device__ __forceinline__ void tile_bounds(uint32_t tile, int cnt, float (&lo)[3],
                                            float (&hi)[3]) {
  lo[0] = lo[1] = lo[2] = 3.0e38f;
  hi[0] = hi[1] = hi[2] = -3.0e38f;
  for (int k = static_cast<int>(threadIdx.x & 31u); k < cnt; k += 32) {
    const float4 p = lds_f4(tile + 16u * k);
    lo[0] = fminf(lo[0], p.x);
    lo[1] = fminf(lo[1], p.y);
    lo[2] = fminf(lo[2], p.z);
    hi[0] = fmaxf(hi[0], p.x);
    hi[1] = fmaxf(hi[1], p.y);
    hi[2] = fmaxf(hi[2], p.z);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], d));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], d));
    }
  }
}

// Whether some (target, source) pair of a tile can be half a box apart on an
// axis: the tile's bounds joined with the targets' (tb = lo[3], hi[3]) span
// at least (1 - 1e-6) L / 2.  If not, every displacement is already its own
// minimum image and the reduction can be skipped (the same bits).
__device__ __forceinline__ bool tile_needs_image(uint32_t tile, int cnt, const float* tb,
                                                 float L) {
  float lo[3], hi[3];
  tile_bounds(tile, cnt, lo, hi);
  const float h = 0.4999995f * L;
  bool need = false;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    need = need || (fmaxf(hi[c], tb[3 + c]) - fminf(lo[c], tb[c]) >= h);
  return need;
}

// Bounds of a CTA's targets into tb[6] (shared): lo[3], hi[3].  Every thread
// of the CTA calls it.
template <int THREADS, int R>
__device__ __forceinline__ void target_bounds(const float (&xi)[R], const float (&yi)[R],
                                              const float (&zi)[R], float* tb) {
  static_assert(THREADS % 32 == 0, "whole warps");
  __shared__ float red[THREADS / 32][6];
  float v[6] = {3.0e38f, 3.0e38f, 3.0e38f, -3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    v[0] = fminf(v[0], xi[r]);
    v[1] = fminf(v[1], yi[r]);
    v[2] = fminf(v[2], zi[r]);
    v[3] = fmaxf(v[3], xi[r]);
    v[4] = fmaxf(v[4], yi[r]);
    v[5] = fmaxf(v[5], zi[r]);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c] = fminf(v[c], __shfl_xor_sync(0xffffffffu, v[c], d));
      v[3 + c] = fmaxf(v[3 + c], __shfl_xor_sync(0xffffffffu, v[3 + c], d));
    }
  }
  if ((threadIdx.x & 31u) == 0)
    for (int c = 0; c < 6; ++c) red[threadIdx.x >> 5][c] = v[c];
  __syncthreads();
  if (threadIdx.x < 6) {
    float a = red[0][threadIdx.x];
    for (int k = 1; k < THREADS / 32; ++k)
      a = threadIdx.x < 3 ? fminf(a, red[k][threadIdx.x]) : fmaxf(a, red[k][threadIdx.x]);
    tb[threadIdx.x] = a;
  }
  __syncthreads();
}

// The pairs of one landed tile (the body of sum_sources' tile loop), for
// the minimum-image kernels, which pick MI per tile.
template <int R, bool POT, bool MI>
__device__ __forceinline__ void sum_tile(uint32_t tile, int cnt, const float (&xi)[R],
                                         const float (&yi)[R], const float (&zi)[R], float eps2,
                                         Acc<R, POT>& acc, float L, float invL) {
  float qt;
  if (tile_uniform_q(tile, cnt, qt)) {
    if (qt != 0.0f) {
      int j = 0;
      for (; j + 8 <= cnt; j += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          pair_u<R, POT, MI>(lds_f4(tile + 16u * (j + q)), xi, yi, zi, eps2, acc, L, invL);
        if (POT) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            kahan_add(acc.sp[r], acc.cp[r], __fmul_rn(acc.ap[r], qt));
            acc.ap[r] = 0.0f;
          }
        }
      }
      for (; j < cnt; ++j)
        pair_u<R, POT, MI>(lds_f4(tile + 16u * j), xi, yi, zi, eps2, acc, L, invL);
      fold_q<R, POT>(acc, qt);
    }
  } else {
    int j = 0;
    for (; j + 8 <= cnt; j += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        pair<R, POT, MI>(lds_f4(tile + 16u * (j + q)), xi, yi, zi, eps2, acc, L, invL);
      if (POT) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          kahan_add(acc.sp[r], acc.cp[r], acc.ap[r]);
          acc.ap[r] = 0.0f;
        }
      }
    }
    for (; j < cnt; ++j) pair<R, POT, MI>(lds_f4(tile + 16u * j), xi, yi, zi, eps2, acc, L, invL);
    fold<R, POT>(acc);
  }
}

template <int THREADS, int R, int TILE, int STAGES, bool POT, bool MI = false>
__device__ __forceinline__ bool sum_sources(Stage<TILE, STAGES>& sm, unsigned& it,
                                            const float4* __restrict__ src, long long ns,
                                            const float (&xi)[R], const float (&yi)[R],
                                            const float (&zi)[R], float eps2, Acc<R, POT>& acc,
                                            int* err, int* s_abort,
                                            const unsigned char* live = nullptr,
                                            long long gbase = 0, float L = 0.0f,
                                            float invL = 0.0f, const float* tb = nullptr) {
  const int ntiles = static_cast<int>((ns + TILE - 1) / TILE);
  // consumers and the issuing thread walk the same sequence of live tiles;
  // the k-th live tile goes through ring stage (it + k) % STAGES
  int t = next_live_tile(live, gbase, ns, 0, ntiles, TILE);
  int ti = t;          // issue cursor (thread 0)
  unsigned issued = 0;
  if (threadIdx.x == 0) {
    for (; issued < static_cast<unsigned>(STAGES) && ti < ntiles; ++issued) {
      issue_tile<TILE, STAGES>(sm, it + issued, src, ns, ti);
      ti = next_live_tile(live, gbase, ns, ti + 1, ntiles, TILE);
    }
  }
  unsigned k = 0;
  for (; t < ntiles; ++k) {
    const unsigned g = it + k;
    const int s = static_cast<int>(g % STAGES);
    const uint32_t parity = (g / STAGES) & 1u;
    if (!mbar_wait(&sm.full[s], parity)) {
      atomicOr(err, kErrTimeout);
      *s_abort = 1;
    }
    if (!*reinterpret_cast<volatile int*>(s_abort)) {
      const uint32_t tile = smem_u32(&sm.tile[s][0]);
      const long long rem = ns - static_cast<long long>(t) * TILE;
      const int cnt = static_cast<int>(rem < TILE ? rem : TILE);
      if constexpr (MI) {
        // a tile whose pairs all lie within half a box needs no image: the
        // plain sum gives the same bits
        if (tile_needs_image(tile, cnt, tb, L))
          sum_tile<R, POT, true>(tile, cnt, xi, yi, zi, eps2, acc, L, invL);
        else
          sum_tile<R, POT, false>(tile, cnt, xi, yi, zi, eps2, acc, L, invL);
      } else {
        float qt;
        if (tile_uniform_q(tile, cnt, qt)) {
          // one charge for the whole tile (records are grouped by species);
          // an uncharged tile adds nothing
          if (qt != 0.0f) {
            int j = 0;
            for (; j + 8 <= cnt; j += 8) {
#pragma unroll
              for (int q = 0; q < 8; ++q)
                pair_u<R, POT, MI>(lds_f4(tile + 16u * (j + q)), xi, yi, zi, eps2, acc, L, invL);
              if (POT) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                  kahan_add(acc.sp[r], acc.cp[r], __fmul_rn(acc.ap[r], qt));
                  acc.ap[r] = 0.0f;
                }
              }
            }
            for (; j < cnt; ++j)
              pair_u<R, POT, MI>(lds_f4(tile + 16u * j), xi, yi, zi, eps2, acc, L, invL);
            fold_q<R, POT>(acc, qt);
          }
        } else {
          int j = 0;
          for (; j + 8 <= cnt; j += 8) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              pair<R, POT, MI>(lds_f4(tile + 16u * (j + q)), xi, yi, zi, eps2, acc, L, invL);
            if (POT) {
              // potential terms of one species share a sign: fold them often so
              // the FP32 partial stays small against a cancelling total
#pragma unroll
              for (int r = 0; r < R; ++r) {
                kahan_add(acc.sp[r], acc.cp[r], acc.ap[r]);
                acc.ap[r] = 0.0f;
              }
            }
          }
          for (; j < cnt; ++j)
            pair<R, POT, MI>(lds_f4(tile + 16u * j), xi, yi, zi, eps2, acc, L, invL);
          fold<R, POT>(acc);
        }
      }
    }
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(s_abort)) {
      if (threadIdx.x == 0) {
        // wait (bounded) for the copies still in flight before leaving
        for (unsigned q = k + 1; q < issued; ++q) {
          const unsigned gq = it + q;
          mbar_wait(&sm.full[gq % STAGES], (gq / STAGES) & 1u);
        }
      }
      __syncthreads();
      return false;
    }
    if (threadIdx.x == 0 && ti < ntiles) {
      issue_tile<TILE, STAGES>(sm, it + issued, src, ns, ti);
      ++issued;
      ti = next_live_tile(live, gbase, ns, ti + 1, ntiles, TILE);
    }
    t = next_live_tile(live, gbase, ns, t + 1, ntiles, TILE);
  }
  it += k;
  return true;
}

// ------------------------------------------------ packed (f32x2) pair path --
//
// sm_100-family packed FP32: add/sub/mul/fma.rn.f32x2 apply the scalar IEEE
// operation to two lanes held in one 64-bit register pair.  Two i-particles
// share each instruction, halving the issue slots per pair (12 packed FP32
// instructions and 2 MUFU per two pairs) while the FMA pipe does the same lane
// work; the per-lane results are bit-identical to the scalar path.

using u64 = unsigned long long;

__device__ __forceinline__ u64 f2_pack(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 f2_add(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 f2_sub(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 f2_mul(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 f2_fma(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ void kahan_add2(u64& s, u64& c, u64 v) {
  const u64 y = f2_sub(v, c);
  const u64 t = f2_add(s, y);
  c = f2_sub(f2_sub(t, s), y);
  s = t;
}

// min_image of both lanes: mi = (-L, 1/L, 1.5 2^23) packed; the same three
// rounded operations per lane as the scalar min_image.
__device__ __forceinline__ u64 f2_min_image(u64 d, const u64 (&mi)[3]) {
  const u64 k = f2_sub(f2_fma(d, mi[1], mi[2]), mi[2]);
  return f2_fma(mi[0], k, d);
}

// A tile of sources expanded for packed use: per source (x,x | y,y) and
// (z,z | q,q), so one LDS.128 yields two ready register pairs.
template <int TILE>
struct DupTile {
  alignas(16) ulonglong2 v[TILE][2];
};

template <int P, bool POT>
struct AccP {
  u64 ax[P], ay[P], az[P], ap[P];  // packed FP32 partials of the current tile
};

// Kahan sums and compensations of the packed path, one slot per thread, kept
// in shared memory (folded once per tile) so the registers hold only the
// targets and the tile partials: [component][pair][thread], component =
// sx, sy, sz, cx, cy, cz (, sp, cp with the potential).  t holds each
// thread's packed targets (x, y, z of its target pairs) and, in e2, the
// packed softening: the source loop reads them back once per unit, so ptxas
// keeps them as loaded register pairs instead of rebuilding each pair from
// its two scalar halves at every use (two ALU moves per use, measured as ~3
// ALU instructions per pair).
template <int P, int THREADS, bool POT>
struct KahanSmem {
  u64 v[POT ? 8 : 6][P][THREADS];
  u64 t[3][P][THREADS];
  u64 e2[THREADS];
};

__device__ __forceinline__ u64 lds_u64(uint32_t addr) {
  u64 v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}

// Component k (0..5: sx, sy, sz, cx, cy, cz) of target r of this thread.
template <int P, int THREADS, bool POT>
__device__ __forceinline__ float kahan_part(const KahanSmem<P, THREADS, POT>& ks, int k, int r) {
  float lo, hi;
  f2_unpack(ks.v[k][r >> 1][threadIdx.x], lo, hi);
  return (r & 1) ? hi : lo;
}

template <int P, bool POT, bool IMG = false>
__device__ __forceinline__ void pair2(const ulonglong2 xy, const ulonglong2 zq, const u64 (&xi)[P],
                                      const u64 (&yi)[P], const u64 (&zi)[P], u64 e2,
                                      AccP<P, POT>& a, const u64 (&mi)[3]) {
#pragma unroll
  for (int p = 0; p < P; ++p) {
    u64 dx = f2_sub(xy.x, xi[p]);
    u64 dy = f2_sub(xy.y, yi[p]);
    u64 dz = f2_sub(zq.x, zi[p]);
    if constexpr (IMG) {
      dx = f2_min_image(dx, mi);
      dy = f2_min_image(dy, mi);
      dz = f2_min_image(dz, mi);
    }
    u64 r2 = f2_fma(dx, dx, e2);
    r2 = f2_fma(dy, dy, r2);
    r2 = f2_fma(dz, dz, r2);
    float lo, hi;
    f2_unpack(r2, lo, hi);
    const u64 ri = f2_pack(rsqrt_mufu(lo), rsqrt_mufu(hi));
    const u64 qr = f2_mul(zq.y, ri);
    const u64 ri2 = f2_mul(ri, ri);
    const u64 s = f2_mul(qr, ri2);
    a.ax[p] = f2_fma(dx, s, a.ax[p]);
    a.ay[p] = f2_fma(dy, s, a.ay[p]);
    a.az[p] = f2_fma(dz, s, a.az[p]);
    if (POT) a.ap[p] = f2_add(a.ap[p], qr);
  }
}

// pair2 for a tile of one charge (see pair_u): no charge multiply per pair.
template <int P, bool POT, bool IMG = false>
__device__ __forceinline__ void pair2_u(const ulonglong2 xy, const ulonglong2 zq,
                                        const u64 (&xi)[P], const u64 (&yi)[P],
                                        const u64 (&zi)[P], u64 e2, AccP<P, POT>& a,
                                        const u64 (&mi)[3]) {
#pragma unroll
  for (int p = 0; p < P; ++p) {
    u64 dx = f2_sub(xy.x, xi[p]);
    u64 dy = f2_sub(xy.y, yi[p]);
    u64 dz = f2_sub(zq.x, zi[p]);
    if constexpr (IMG) {
      dx = f2_min_image(dx, mi);
      dy = f2_min_image(dy, mi);
      dz = f2_min_image(dz, mi);
    }
    u64 r2 = f2_fma(dx, dx, e2);
    r2 = f2_fma(dy, dy, r2);
    r2 = f2_fma(dz, dz, r2);
    float lo, hi;
    f2_unpack(r2, lo, hi);
    const u64 ri = f2_pack(rsqrt_mufu(lo), rsqrt_mufu(hi));
    const u64 ri2 = f2_mul(ri, ri);
    const u64 s = f2_mul(ri2, ri);
    a.ax[p] = f2_fma(dx, s, a.ax[p]);
    a.ay[p] = f2_fma(dy, s, a.ay[p]);
    a.az[p] = f2_fma(dz, s, a.az[p]);
    if (POT) a.ap[p] = f2_add(a.ap[p], ri);
  }
}

// As sum_sources, with the pair arithmetic in packed f32x2.  Each landed
// tile is first expanded into `dup` (which frees its TMA stage at once, so a
// single stage suffices), then the R targets of this thread are summed two at
// a time, four sources per unrolled step (eight were 0.2 % slower and sixteen
// 11 %: the loop's code outgrows the instruction cache).  The Kahan sums live
// in `ks` (bit-identical to the scalar path's); reset = false continues the
// sums of an earlier call instead of clearing them.  MI: as sum_sources, a
// tile some of whose pairs may lie half a box apart (targets' bounds tb)
// takes minimum-image displacements in the cube of side L.
template <int THREADS, int R, int TILE, int STAGES, bool POT, bool MI = false>
__device__ __forceinline__ bool sum_sources_packed(Stage<TILE, STAGES>& sm, DupTile<TILE>& dup,
                                                   KahanSmem<R / 2, THREADS, POT>& ks, unsigned& it,
                                                   const float4* __restrict__ src, long long ns,
                                                   const float (&xi)[R], const float (&yi)[R],
                                                   const float (&zi)[R], float eps2, int* err,
                                                   int* s_abort,
                                                   const unsigned char* live = nullptr,
                                                   long long gbase = 0, bool reset = true,
                                                   float L = 0.0f, float invL = 0.0f,
                                                   const float* tb = nullptr) {
  static_assert(R % 2 == 0, "packed path needs an even number of i-particles per thread");
  constexpr int P = R / 2;
  const int tid = threadIdx.x;
  u64 xi2[P], yi2[P], zi2[P];
  AccP<P, POT> a;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    ks.t[0][p][tid] = f2_pack(xi[2 * p], xi[2 * p + 1]);
    ks.t[1][p][tid] = f2_pack(yi[2 * p], yi[2 * p + 1]);
    ks.t[2][p][tid] = f2_pack(zi[2 * p], zi[2 * p + 1]);
    xi2[p] = lds_u64(smem_u32(&ks.t[0][p][tid]));
    yi2[p] = lds_u64(smem_u32(&ks.t[1][p][tid]));
    zi2[p] = lds_u64(smem_u32(&ks.t[2][p][tid]));
    a.ax[p] = a.ay[p] = a.az[p] = a.ap[p] = 0ull;
    if (reset) {
#pragma unroll
      for (int k = 0; k < (POT ? 8 : 6); ++k) ks.v[k][p][tid] = 0ull;
    }
  }
  ks.e2[tid] = f2_pack(eps2, eps2);
  const u64 e2 = lds_u64(smem_u32(&ks.e2[tid]));
  // MI: the packed minimum-image constants, loaded as register pairs
  u64 mi[3] = {0ull, 0ull, 0ull};
  if constexpr (MI) {
    __shared__ u64 s_mi[3][THREADS];
    s_mi[0][tid] = f2_pack(-L, -L);
    s_mi[1][tid] = f2_pack(invL, invL);
    s_mi[2][tid] = f2_pack(12582912.0f, 12582912.0f);
#pragma unroll
    for (int k = 0; k < 3; ++k) mi[k] = lds_u64(smem_u32(&s_mi[k][tid]));
  }
  const int ntiles = static_cast<int>((ns + TILE - 1) / TILE);
  // live tiles only, in the same order for the issuing thread and the consumers
  int t = next_live_tile(live, gbase, ns, 0, ntiles, TILE);
  int ti = t;
  unsigned issued = 0;
  if (tid == 0) {
    for (; issued < static_cast<unsigned>(STAGES) && ti < ntiles; ++issued) {
      issue_tile<TILE, STAGES>(sm, it + issued, src, ns, ti);
      ti = next_live_tile(live, gbase, ns, ti + 1, ntiles, TILE);
    }
  }
  unsigned kt = 0;
  for (; t < ntiles; ++kt) {
    const unsigned g = it + kt;
    const int s = static_cast<int>(g % STAGES);
    const uint32_t parity = (g / STAGES) & 1u;
    if (!mbar_wait(&sm.full[s], parity)) {
      atomicOr(err, kErrTimeout);
      *s_abort = 1;
    }
    const long long rem = ns - static_cast<long long>(t) * TILE;
    const int cnt = static_cast<int>(rem < TILE ? rem : TILE);
    float qt = 0.0f;
    bool uni = false;
    bool img = false;  // MI: some pair of this tile may be half a box apart
    if (!*reinterpret_cast<volatile int*>(s_abort)) {
      uni = tile_uniform_q(smem_u32(&sm.tile[s][0]), cnt, qt);
      if constexpr (MI) img = tile_needs_image(smem_u32(&sm.tile[s][0]), cnt, tb, L);
      for (int k = tid; k < cnt; k += THREADS) {
        const float4 p = sm.tile[s][k];
        dup.v[k][0] = make_ulonglong2(f2_pack(p.x, p.x), f2_pack(p.y, p.y));
        dup.v[k][1] = make_ulonglong2(f2_pack(p.z, p.z), f2_pack(p.w, p.w));
      }
    }
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(s_abort)) {
      if (tid == 0) {
        for (unsigned q = kt + 1; q < issued; ++q) {
          const unsigned gq = it + q;
          mbar_wait(&sm.full[gq % STAGES], (gq / STAGES) & 1u);
        }
      }
      __syncthreads();
      return false;
    }
    // the stage is expanded into dup: refill it while this tile is summed
    if (tid == 0 && ti < ntiles) {
      issue_tile<TILE, STAGES>(sm, it + issued, src, ns, ti);
      ++issued;
      ti = next_live_tile(live, gbase, ns, ti + 1, ntiles, TILE);
    }
    const uint32_t dbase = smem_u32(&dup.v[0][0]);
    if (uni && qt == 0.0f) {  // an uncharged tile adds nothing
      __syncthreads();
      t = next_live_tile(live, gbase, ns, t + 1, ntiles, TILE);
      continue;
    }
    const u64 qq = f2_pack(qt, qt);
    // the tile's pairs; IMG: with minimum-image displacements
    auto sum_tile2 = [&](auto img_tag) {
      constexpr bool IMG = decltype(img_tag)::value;
      int j = 0;
      if (uni) {
        for (; j + 4 <= cnt; j += 4) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            pair2_u<P, POT, IMG>(lds_u64x2(dbase + 32u * (j + k)),
                                 lds_u64x2(dbase + 32u * (j + k) + 16u), xi2, yi2, zi2, e2, a,
                                 mi);
          if (POT && (j & 4)) {  // the potential is folded every 8 sources
#pragma unroll
            for (int p = 0; p < P; ++p) {
              u64 sp = ks.v[6][p][tid], cp = ks.v[7][p][tid];
              kahan_add2(sp, cp, f2_mul(a.ap[p], qq));
              ks.v[6][p][tid] = sp;
              ks.v[7][p][tid] = cp;
              a.ap[p] = 0ull;
            }
          }
        }
        for (; j < cnt; ++j)
          pair2_u<P, POT, IMG>(lds_u64x2(dbase + 32u * j), lds_u64x2(dbase + 32u * j + 16u), xi2,
                               yi2, zi2, e2, a, mi);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          a.ax[p] = f2_mul(a.ax[p], qq);
          a.ay[p] = f2_mul(a.ay[p], qq);
          a.az[p] = f2_mul(a.az[p], qq);
          if (POT) a.ap[p] = f2_mul(a.ap[p], qq);
        }
      } else {
        for (; j + 4 <= cnt; j += 4) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            pair2<P, POT, IMG>(lds_u64x2(dbase + 32u * (j + k)),
                               lds_u64x2(dbase + 32u * (j + k) + 16u), xi2, yi2, zi2, e2, a,
                               mi);
          if (POT && (j & 4)) {  // the potential is folded every 8 sources
#pragma unroll
            for (int p = 0; p < P; ++p) {
              u64 sp = ks.v[6][p][tid], cp = ks.v[7][p][tid];
              kahan_add2(sp, cp, a.ap[p]);
              ks.v[6][p][tid] = sp;
              ks.v[7][p][tid] = cp;
              a.ap[p] = 0ull;
            }
          }
        }
        for (; j < cnt; ++j)
          pair2<P, POT, IMG>(lds_u64x2(dbase + 32u * j), lds_u64x2(dbase + 32u * j + 16u), xi2, yi2,
                             zi2, e2, a, mi);
      }
    };
    if (MI && img)
      sum_tile2(std::integral_constant<bool, MI>{});
    else
      sum_tile2(std::false_type{});
#pragma unroll
    for (int p = 0; p < P; ++p) {
      u64 sv, cv;
      sv = ks.v[0][p][tid]; cv = ks.v[3][p][tid];
      kahan_add2(sv, cv, a.ax[p]);
      ks.v[0][p][tid] = sv; ks.v[3][p][tid] = cv;
      sv = ks.v[1][p][tid]; cv = ks.v[4][p][tid];
      kahan_add2(sv, cv, a.ay[p]);
      ks.v[1][p][tid] = sv; ks.v[4][p][tid] = cv;
      sv = ks.v[2][p][tid]; cv = ks.v[5][p][tid];
      kahan_add2(sv, cv, a.az[p]);
      ks.v[2][p][tid] = sv; ks.v[5][p][tid] = cv;
      a.ax[p] = a.ay[p] = a.az[p] = 0ull;
      if (POT) {
        sv = ks.v[6][p][tid]; cv = ks.v[7][p][tid];
        kahan_add2(sv, cv, a.ap[p]);
        ks.v[6][p][tid] = sv; ks.v[7][p][tid] = cv;
        a.ap[p] = 0ull;
      }
    }
    __syncthreads();  // dup is rewritten by the next tile
    t = next_live_tile(live, gbase, ns, t + 1, ntiles, TILE);
  }
  it += kt;
  return true;
}

// ------------------------------------------------------------ step kernel --

// Ion energy detectors.  The decisions (crossing, cone, energy bin) are FP64
// with every operation rounded to nearest in the order written, no
// contraction, so they are taken exactly as a plain sequential program takes
// them from the same numbers.
constexpr double kDetMeC2Ev = 510998.95;

__device__ __forceinline__ double det_norm2(double a, double b, double c) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// (gamma - 1) m c^2 in eV, as u^2/(sqrt(1 + u^2) + 1) m c^2.
__device__ __forceinline__ double det_ke_ev(double ux, double uy, double uz, double mass) {
  const double uu = det_norm2(ux, uy, uz);
  const double g1 = __ddiv_rn(uu, __dadd_rn(__dsqrt_rn(__dadd_rn(1.0, uu)), 1.0));
  return __dmul_rn(__dmul_rn(g1, mass), kDetMeC2Ev);
}

__device__ __forceinline__ int det_bin(double ke, double emax, int nbins) {
  if (!(ke < emax)) return nbins;
  const int b = static_cast<int>(floor(__ddiv_rn(__dmul_rn(ke, static_cast<double>(nbins)), emax)));
  return b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
}

// Records ion i if it crossed the detector sphere outward in this step:
// histograms +x, -x, +y, -y (cone of half-angle acos(det_cos)) and all.
// Compiled only into the step kernels instantiated with detectors: present in
// the epilogue, even behind a branch that is never taken, it changes the code
// of the whole kernel (2.6 % slower).
__device__ __forceinline__ void detect(unsigned long long* hist, unsigned char* crossed,
                                       const ClusterDev& c, long long i, double x0, double y0,
                                       double z0, double x1, double y1, double z1, double ux,
                                       double uy, double uz, double mass, int* err) {
  if (crossed[i]) return;
  const double rp2 = det_norm2(__dsub_rn(x0, c.det_c[0]), __dsub_rn(y0, c.det_c[1]),
                               __dsub_rn(z0, c.det_c[2]));
  const double b0 = __dsub_rn(x1, c.det_c[0]), b1 = __dsub_rn(y1, c.det_c[1]);
  const double rn2 = det_norm2(b0, b1, __dsub_rn(z1, c.det_c[2]));
  if (!(rp2 < c.det_r2 && rn2 >= c.det_r2)) return;
  crossed[i] = 1;
  const int nb1 = c.det_nbins + 1;
  const int bin = det_bin(det_ke_ev(ux, uy, uz, mass), c.det_emax, c.det_nbins);
  if (!MD_IN_RANGE(err, bin, 0, c.det_nbins + 1)) return;
  const double cc = __dmul_rn(c.det_cos, __dsqrt_rn(rn2));
  unsigned long long* h = hist + c.det_off;
  atomicAdd(h + 4 * nb1 + bin, 1ull);
  if (b0 >= cc) atomicAdd(h + 0 * nb1 + bin, 1ull);
  if (-b0 >= cc) atomicAdd(h + 1 * nb1 + bin, 1ull);
  if (b1 >= cc) atomicAdd(h + 2 * nb1 + bin, 1ull);
  if (-b1 >= cc) atomicAdd(h + 3 * nb1 + bin, 1ull);
}

// Laser + Boris kick (FP32 increment) + FP64 drift + boundary for record i
// with Coulomb field (ex, ey, ez); writes x, u and the next j-stream entry.
// DIAG (diagnostic steps): also the record's diagnostics at t_n, as
// k_diag_partial forms them from the same kick: status (1 active, 2
// non-finite; inactive records are left at 0), kinetic energy at the
// integer-time u = u^{n-1/2} + du/2, potential energy w z phi / 2, momentum.
template <bool DET, bool DIAG = false>
__device__ __forceinline__ void push_record(const StepArgs& a, const ClusterDev& c, long long i,
                                            double ex, double ey, double ez, const float* las,
                                            double t_next, const float4* cur, float4* nxt,
                                            double phi = 0.0) {
  if (!MD_IN_RANGE(a.err, i, c.off, c.off + c.n_pad)) return;
  double X = a.x[i], Y = a.y[i], Z = a.z[i];
  double Ux = a.ux[i], Uy = a.uy[i], Uz = a.uz[i];
  const float h = 0.5f * static_cast<float>(c.dt) * a.qm[i];
  float dux, duy, duz;
  boris_increment(static_cast<float>(Ux), static_cast<float>(Uy), static_cast<float>(Uz),
                  static_cast<float>(ex) + las[0], static_cast<float>(ey) + las[1],
                  static_cast<float>(ez) + las[2], las[3], las[4], las[5], h, dux, duy, duz);
  if constexpr (DIAG) {
    if (a.kind[i] != 2) {
      double* rec = a.diag_rec + 6 * i;
      if (!(isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(Ux) && isfinite(Uy) &&
            isfinite(Uz))) {
        rec[0] = 2.0;
      } else {
        const double mx = Ux + 0.5 * dux, my = Uy + 0.5 * duy, mz = Uz + 0.5 * duz;
        const double uu = mx * mx + my * my + mz * mz;
        const double wm = a.w[i] * a.mass[i];
        rec[0] = 1.0;
        rec[1] = wm * uu / (sqrt(1.0 + uu) + 1.0);
        rec[2] = 0.5 * a.w[i] * a.zq[i] * phi;
        rec[3] = wm * mx;
        rec[4] = wm * my;
        rec[5] = wm * mz;
      }
    }
  }
  Ux += static_cast<double>(dux);
  Uy += static_cast<double>(duy);
  Uz += static_cast<double>(duz);
  const double ginv = rsqrt(1.0 + (Ux * Ux + Uy * Uy + Uz * Uz));
  X += c.dt * Ux * ginv;
  Y += c.dt * Uy * ginv;
  Z += c.dt * Uz * ginv;
  const bool wrap = (c.boundary == 1) || (c.boundary == 2 && t_next < c.t_switch);
  if (wrap) {
    X = wrap_periodic(X, c.box);
    Y = wrap_periodic(Y, c.box);
    Z = wrap_periodic(Z, c.box);
  }
  if constexpr (DET) {
    if (c.det_nbins > 0 && a.det_hist && a.qm[i] > 0.0f)
      detect(a.det_hist, a.det_crossed, c, i, a.x[i], a.y[i], a.z[i], X, Y, Z, Ux, Uy, Uz,
             a.mass[i], a.err);
  }
  a.x[i] = X;
  a.y[i] = Y;
  a.z[i] = Z;
  a.ux[i] = Ux;
  a.uy[i] = Uy;
  a.uz[i] = Uz;
  nxt[i] = make_float4(static_cast<float>(X), static_cast<float>(Y), static_cast<float>(Z),
                       cur[i].w);
  if (a.vel) {
    float4 v = a.vel[i];
    v.x = static_cast<float>(Ux);
    v.y = static_cast<float>(Uy);
    v.z = static_cast<float>(Uz);
    a.vel[i] = v;
  }
}

// Sum of the n partials p[k stride] (C components each, k = 0 .. n - 1) of
// one target, added in index order; the loads of kInFlight partials are
// issued before their adds, so the sum costs n / kInFlight round trips to L2.
template <int C, int kInFlight>
__device__ __forceinline__ void sum_partials(const double* p, long long stride, int n, double& x,
                                             double& y, double& z) {
  x = 0.0;
  y = 0.0;
  z = 0.0;
#pragma unroll 1
  for (int k0 = 0; k0 < n; k0 += kInFlight) {
    double v[kInFlight][C];
#pragma unroll
    for (int k = 0; k < kInFlight; ++k)
      if (k0 + k < n) {
#pragma unroll
        for (int c = 0; c < C; ++c) v[k][c] = __ldcg(p + (k0 + k) * stride + c);
      }
#pragma unroll
    for (int k = 0; k < kInFlight; ++k)
      if (k0 + k < n) {
        x += v[k][0];
        if constexpr (C > 1) {
          y += v[k][1];
          z += v[k][2];
        }
      }
  }
}

// One full MD step for every work unit (cluster, i-block, piece): field at x^n
// from the piece's sources, and once all pieces of an i-block are summed,
// laser at t_n, Boris kick, FP64 drift, boundary, new j-stream entry.
// Persistent: CTAs take shares (runs of units) from an atomic ticket.
//
// POT: a diagnostic step, which also sums the potential phi_i beside the
// field (split pieces add their phi partials in order) and records every
// record's diagnostics at t_n (push_record's DIAG).
//
// MI: clusters whose min_image flag is set sum minimum-image displacements
// while their boundary is periodic.
template <int THREADS, int R, int TILE, int STAGES, bool PACK, int MINB, bool DET,
          bool POT = false, bool MI = false>
__global__ void __launch_bounds__(THREADS, MINB) k_step(const StepArgs a) {
  __shared__ Stage<TILE, STAGES> sm;
  __shared__ DupTile<PACK ? TILE : 1> dup;
  __shared__ KahanSmem<PACK ? R / 2 : 1, PACK ? THREADS : 1, POT> ks;
  __shared__ int s_unit, s_abort, s_last;
  __shared__ float s_las[6];
  // the current unit's cluster and ranges live in shared memory, not in
  // registers, so that nothing but the targets and partials is held across
  // the source loop
  __shared__ ClusterDev s_c;
  __shared__ Unit s_un;

  const long long step = __ldcg(a.step);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();

  unsigned it = 0;
  for (;;) {
    if (threadIdx.x == 0) s_unit = static_cast<int>(atomicAdd(a.ticket, 1u));
    __syncthreads();
    const int share = s_unit;
    __syncthreads();  // s_unit is rewritten by the next share's ticket
    if (share >= a.n_shares) break;
    const int u_end = a.share_first[share + 1];
#pragma unroll 1
    for (int u = a.share_first[share]; u < u_end; ++u) {
      if (threadIdx.x == 0) {
        s_un = a.units[u];
        s_c = a.cl[s_un.cluster];
        laser_field(s_c, s_c.t0 + static_cast<double>(step) * s_c.dt, s_las);
      }
      __syncthreads();
      if (any_live(a.tgt_live, s_c.off + static_cast<long long>(s_un.block) * (THREADS * R),
                   (s_c.off + static_cast<long long>(s_un.block + 1) * (THREADS * R) <
                            s_c.off + s_c.n_pad
                        ? s_c.off + static_cast<long long>(s_un.block + 1) * (THREADS * R)
                        : s_c.off + s_c.n_pad) - 1)) {
        const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
        const long long i0 = s_c.off + static_cast<long long>(s_un.block) * (THREADS * R);
        const long long iend = s_c.off + s_c.n_pad;
        long long j0, jn;
        if (s_un.jn >= 0) {
          j0 = s_un.j0;
          jn = s_un.jn;
          if (!MD_IN_RANGE(a.err, j0 + jn, 1, s_c.n_pad + 1)) jn = 0;  // a piece in the cluster
        } else {
          j0 = static_cast<long long>(s_un.seg) * s_c.seg_len;
          const long long jrem = s_c.n_pad - j0;
          jn = jrem < s_c.seg_len ? jrem : s_c.seg_len;
        }
        float xi[R], yi[R], zi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const long long i = i0 + threadIdx.x + r * THREADS;
          const float4 p = (i < iend) ? cur[i] : make_float4(0.f, 0.f, 0.f, 0.f);
          xi[r] = p.x;
          yi[r] = p.y;
          zi[r] = p.z;
        }
        bool ok;
        Acc<R, POT> acc;
        // MI: minimum-image forces while this cluster's boundary is periodic at t_n
        bool mi = false;
        if constexpr (MI) {
          const double t_n = s_c.t0 + static_cast<double>(step) * s_c.dt;
          mi = a.min_image && a.min_image[s_un.cluster] &&
               (s_c.boundary == 1 || (s_c.boundary == 2 && t_n < s_c.t_switch));
        }
        if constexpr (PACK) {
          if (MI && mi) {
            __shared__ float s_tb2[6];  // bounds of this unit's targets
            target_bounds<THREADS, R>(xi, yi, zi, s_tb2);
            const float L = static_cast<float>(s_c.box);
            ok = sum_sources_packed<THREADS, R, TILE, STAGES, POT, MI>(
                sm, dup, ks, it, cur + s_c.off + j0, jn, xi, yi, zi, s_c.eps2, a.err, &s_abort,
                a.src_live, s_c.off + j0, true, L, 1.0f / L, s_tb2);
          } else {
            ok = sum_sources_packed<THREADS, R, TILE, STAGES, POT>(
                sm, dup, ks, it, cur + s_c.off + j0, jn, xi, yi, zi, s_c.eps2, a.err, &s_abort,
                a.src_live, s_c.off + j0);
          }
        } else {
          acc.zero();
          if constexpr (MI) {
            if (mi) {
              __shared__ float s_tb[6];  // bounds of this unit's targets
              target_bounds<THREADS, R>(xi, yi, zi, s_tb);
              const float L = static_cast<float>(s_c.box);
              ok = sum_sources<THREADS, R, TILE, STAGES, POT, true>(
                  sm, it, cur + s_c.off + j0, jn, xi, yi, zi, s_c.eps2, acc, a.err, &s_abort,
                  a.src_live, s_c.off + j0, L, 1.0f / L, s_tb);
            } else {
              ok = sum_sources<THREADS, R, TILE, STAGES, POT>(
                  sm, it, cur + s_c.off + j0, jn, xi, yi, zi, s_c.eps2, acc, a.err, &s_abort,
                  a.src_live, s_c.off + j0);
            }
          } else {
            ok = sum_sources<THREADS, R, TILE, STAGES, POT>(sm, it, cur + s_c.off + j0, jn, xi, yi,
                                                            zi, s_c.eps2, acc, a.err, &s_abort,
                                                            a.src_live, s_c.off + j0);
          }
        }
        if (!ok) return;

        // field at target r: -(Kahan total s - c) of sum Q (x_j - x_i)/r^3
        auto field_of = [&](int r, double& ex, double& ey, double& ez) {
          if constexpr (PACK) {
            ex = -(static_cast<double>(kahan_part(ks, 0, r)) - kahan_part(ks, 3, r));
            ey = -(static_cast<double>(kahan_part(ks, 1, r)) - kahan_part(ks, 4, r));
            ez = -(static_cast<double>(kahan_part(ks, 2, r)) - kahan_part(ks, 5, r));
          } else {
            ex = -(static_cast<double>(acc.sx[r]) - acc.cx[r]);
            ey = -(static_cast<double>(acc.sy[r]) - acc.cy[r]);
            ez = -(static_cast<double>(acc.sz[r]) - acc.cz[r]);
          }
        };
        // POT: the potential's Kahan total (s - c) at target r
        auto phi_of = [&](int r) -> double {
          if constexpr (PACK && POT)
            return static_cast<double>(kahan_part(ks, 6, r)) - kahan_part(ks, 7, r);
          else if constexpr (POT)
            return static_cast<double>(acc.sp[r]) - acc.cp[r];
          else
            return 0.0;
        };

        // the unit's ranges are re-read from shared memory after the loop
        const float4* __restrict__ cur2 = (step & 1) ? a.posq1 : a.posq0;
        float4* __restrict__ nxt = (step & 1) ? a.posq0 : a.posq1;
        const long long e0 = s_c.off + static_cast<long long>(s_un.block) * (THREADS * R);
        const long long eend = s_c.off + s_c.n_pad;
        const double t_next = s_c.t0 + static_cast<double>(step + 1) * s_c.dt;
        const int nparts = s_un.jn >= 0 ? s_un.nparts : s_c.nseg;
        if (nparts == 1) {
          // the packed path reads its sums from shared memory, so its epilogue
          // stays rolled (one FP64 push at a time)
          if constexpr (PACK) {
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
              const long long i = e0 + threadIdx.x + r * THREADS;
              if (i >= eend) continue;
              double ex, ey, ez;
              field_of(r, ex, ey, ez);
              if constexpr (POT) {
                const double ph =
                    phi_of(r) - static_cast<double>(cur2[i].w * rsqrt_mufu(s_c.eps2));
                push_record<DET, true>(a, s_c, i, ex, ey, ez, s_las, t_next, cur2, nxt, ph);
              } else {
                push_record<DET>(a, s_c, i, ex, ey, ez, s_las, t_next, cur2, nxt);
              }
            }
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const long long i = e0 + threadIdx.x + r * THREADS;
              if (i >= eend) continue;
              double ex, ey, ez;
              field_of(r, ex, ey, ez);
              if constexpr (POT) {
                // the potential without the record's own term
                const double ph =
                    phi_of(r) - static_cast<double>(cur2[i].w * rsqrt_mufu(s_c.eps2));
                push_record<DET, true>(a, s_c, i, ex, ey, ez, s_las, t_next, cur2, nxt, ph);
              } else {
                push_record<DET>(a, s_c, i, ex, ey, ez, s_las, t_next, cur2, nxt);
              }
            }
          }
        } else {
          // this unit covers one piece of the sources: publish the partial
          // field; the last of the nparts units of this i-block sums the
          // partials in piece order (deterministic) and pushes
          const int seg = s_un.seg;
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const long long i = e0 + threadIdx.x + r * THREADS;
            if (i >= eend) continue;
            double ex, ey, ez;
            field_of(r, ex, ey, ez);
            if (!MD_IN_RANGE(a.err, seg, 0, nparts) || !MD_IN_RANGE(a.err, i, 0, a.n_total))
              continue;
            double* p = a.part + 3 * (static_cast<long long>(seg) * a.n_total + i);
            __stcg(p + 0, ex);
            __stcg(p + 1, ey);
            __stcg(p + 2, ez);
            if constexpr (POT)
              __stcg(a.part_phi + static_cast<long long>(seg) * a.n_total + i, phi_of(r));
          }
          __threadfence();
          __syncthreads();
          if (threadIdx.x == 0) {
            const unsigned prev = atomicAdd(a.iblk_cnt + s_un.ib, 1u);
            s_last = (prev == static_cast<unsigned>(nparts - 1));
            if (s_last) atomicExch(a.iblk_cnt + s_un.ib, 0u);
          }
          __syncthreads();
          if (s_last) {
            __threadfence();
            const int nseg = nparts;
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
              const long long i = e0 + threadIdx.x + r * THREADS;
              if (i >= eend) continue;
              // eight partials in flight on the packed path (measured 2-3 %
              // faster at 100k-400k records with 4 equal shares per CTA, the
              // ptxas register budget rising with it), one on the scalar path
              double ex, ey, ez;
              sum_partials<3, PACK ? 8 : 1>(a.part + 3 * i, 3 * a.n_total, nseg, ex, ey, ez);
              if constexpr (POT) {
                double ph, d1, d2;
                sum_partials<1, 1>(a.part_phi + i, a.n_total, nseg, ph, d1, d2);
                ph -= static_cast<double>(cur2[i].w * rsqrt_mufu(s_c.eps2));
                push_record<DET, true>(a, s_c, i, ex, ey, ez, s_las, t_next, cur2, nxt, ph);
              } else {
                push_record<DET>(a, s_c, i, ex, ey, ez, s_las, t_next, cur2, nxt);
              }
            }
          }
        }
      }
      __syncthreads();
    }
  }

  // last CTA out: reset the ticket, advance the step counter
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(a.done, 1u);
    if (prev == gridDim.x - 1) {
      atomicExch(a.ticket, 0u);
      atomicExch(a.done, 0u);
      __threadfence();
      *reinterpret_cast<volatile long long*>(a.step) = step + 1;
    }
  }
}

// ----------------------------------------------------------- field kernel --

// Field (and potential) at targets from sources; one target block per CTA.
template <int THREADS, int R, int TILE, int STAGES, bool POT, bool MI = false, bool PACK = false>
__global__ void __launch_bounds__(THREADS) k_field(const FieldArgs a) {
  __shared__ Stage<TILE, STAGES> sm;
  __shared__ DupTile<PACK ? TILE : 1> dup;
  __shared__ KahanSmem<PACK ? R / 2 : 1, PACK ? THREADS : 1, POT> ks;
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  // this CTA's sources: all, or segment blockIdx.y of a split
  const bool split = a.nseg > 1;
  const long long j0 = split ? static_cast<long long>(blockIdx.y) * a.seg_len : 0;
  const long long jn = split ? (a.ns - j0 < a.seg_len ? (a.ns > j0 ? a.ns - j0 : 0) : a.seg_len)
                             : a.ns;
  double* part = split ? a.part + 4 * static_cast<long long>(blockIdx.y) * a.nt : nullptr;
  const long long i0 = static_cast<long long>(blockIdx.x) * (THREADS * R);
  const long long i1 = (i0 + THREADS * R < a.nt ? i0 + THREADS * R : a.nt) - 1;
  if (a.tgt_live && !any_live(a.tgt_live, a.gbase + i0, a.gbase + i1)) {
    // no active record among these targets: zero field and potential
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const long long i = i0 + threadIdx.x + r * THREADS;
      if (i >= a.nt) continue;
      if (split) {
        part[4 * i + 0] = part[4 * i + 1] = part[4 * i + 2] = part[4 * i + 3] = 0.0;
        continue;
      }
      a.e[3 * i + 0] = a.e[3 * i + 1] = a.e[3 * i + 2] = 0.0;
      if (POT && a.phi) a.phi[i] = 0.0;
    }
    return;
  }
  float xi[R], yi[R], zi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = i0 + threadIdx.x + r * THREADS;
    const float4 p = (i < a.nt) ? a.tgt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
  }
  Acc<R, POT> acc;
  acc.zero();
  unsigned it = 0;
  bool ok;
  if constexpr (PACK) {
    __shared__ float s_tb[6];  // bounds of this CTA's targets
    if constexpr (MI) target_bounds<THREADS, R>(xi, yi, zi, s_tb);
    ok = sum_sources_packed<THREADS, R, TILE, STAGES, POT, MI>(
        sm, dup, ks, it, a.src + j0, jn, xi, yi, zi, a.eps2, a.err, &s_abort, a.src_live,
        a.gbase + j0, true, a.box, MI ? 1.0f / a.box : 0.0f, s_tb);
  } else if constexpr (MI) {
    __shared__ float s_tb[6];  // bounds of this CTA's targets
    target_bounds<THREADS, R>(xi, yi, zi, s_tb);
    ok = sum_sources<THREADS, R, TILE, STAGES, POT, true>(sm, it, a.src + j0, jn, xi, yi, zi,
                                                          a.eps2, acc, a.err, &s_abort,
                                                          a.src_live, a.gbase + j0, a.box,
                                                          1.0f / a.box, s_tb);
  } else {
    ok = sum_sources<THREADS, R, TILE, STAGES, POT>(sm, it, a.src + j0, jn, xi, yi, zi, a.eps2,
                                                    acc, a.err, &s_abort, a.src_live,
                                                    a.gbase + j0);
  }
  if (!ok) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = i0 + threadIdx.x + r * THREADS;
    if (i >= a.nt) continue;
    double ex, ey, ez, ph = 0.0;
    if constexpr (PACK) {
      ex = -(static_cast<double>(kahan_part(ks, 0, r)) - kahan_part(ks, 3, r));
      ey = -(static_cast<double>(kahan_part(ks, 1, r)) - kahan_part(ks, 4, r));
      ez = -(static_cast<double>(kahan_part(ks, 2, r)) - kahan_part(ks, 5, r));
      if constexpr (POT) ph = static_cast<double>(kahan_part(ks, 6, r)) - kahan_part(ks, 7, r);
    } else {
      ex = -(static_cast<double>(acc.sx[r]) - acc.cx[r]);
      ey = -(static_cast<double>(acc.sy[r]) - acc.cy[r]);
      ez = -(static_cast<double>(acc.sz[r]) - acc.cz[r]);
      if constexpr (POT) ph = static_cast<double>(acc.sp[r]) - acc.cp[r];
    }
    if (split) {
      part[4 * i + 0] = ex;
      part[4 * i + 1] = ey;
      part[4 * i + 2] = ez;
      part[4 * i + 3] = ph;
      continue;
    }
    a.e[3 * i + 0] = ex;
    a.e[3 * i + 1] = ey;
    a.e[3 * i + 2] = ez;
    if (POT && a.phi) {
      if (a.self_offset >= 0) {
        const long long js = i + a.self_offset;
        if (js < a.ns) ph -= static_cast<double>(a.src[js].w * rsqrt_mufu(a.eps2));
      }
      a.phi[i] = ph;
    }
  }
}

// ------------------------------------------------------- diagnostics (K4) --

template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < THREADS / 32; ++k) s += red[k];
  return s;  // valid in thread 0
}

// Per-block FP64 partial sums of the diagnostics of one cluster.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_diag_partial(const DiagArgs a) {
  __shared__ double red[THREADS / 32];
  const long long step = __ldcg(a.step);
  const double t_n = a.c.t0 + static_cast<double>(step) * a.c.dt;
  float las[6];
  laser_field(a.c, t_n, las);
  const float hq = 0.5f * static_cast<float>(a.c.dt);
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long na = 0, nbad = 0;
  long long hist[kHistBins];
  double histw[kHistBins];
#pragma unroll
  for (int k = 0; k < kHistBins; ++k) {
    hist[k] = 0;
    histw[k] = 0.0;
  }
  for (long long k = static_cast<long long>(blockIdx.x) * THREADS + threadIdx.x; k < a.c.n;
       k += static_cast<long long>(gridDim.x) * THREADS) {
    const long long i = a.c.off + k;
    const unsigned char kd = a.kind[i];
    if (kd == 2) continue;
    ++na;
    if (a.rec) {
      // recorded by a diagnostic step at t_n (the state here is t_{n+1})
      const double* rc = a.rec + 6 * i;
      if (rc[0] != 1.0) {
        ++nbad;
        continue;
      }
      acc[0] += rc[1];
      if (kd == 1) acc[2] += rc[1]; else acc[1] += rc[1];
      acc[3] += rc[2];
      acc[4] += rc[3];
      acc[5] += rc[4];
      acc[6] += rc[5];
    } else {
      const double X = a.x[i], Y = a.y[i], Z = a.z[i];
      const double Ux = a.ux[i], Uy = a.uy[i], Uz = a.uz[i];
      if (!(isfinite(X) && isfinite(Y) && isfinite(Z) && isfinite(Ux) && isfinite(Uy) &&
            isfinite(Uz))) {
        ++nbad;
        continue;
      }
      float dux, duy, duz;
      boris_increment(static_cast<float>(Ux), static_cast<float>(Uy), static_cast<float>(Uz),
                      static_cast<float>(a.e[3 * k]) + las[0],
                      static_cast<float>(a.e[3 * k + 1]) + las[1],
                      static_cast<float>(a.e[3 * k + 2]) + las[2], las[3], las[4], las[5],
                      hq * a.qm[i], dux, duy, duz);
      const double mx = Ux + 0.5 * dux, my = Uy + 0.5 * duy, mz = Uz + 0.5 * duz;
      const double uu = mx * mx + my * my + mz * mz;
      const double wm = a.w[i] * a.mass[i];
      const double ke = wm * uu / (sqrt(1.0 + uu) + 1.0);
      acc[0] += ke;
      if (kd == 1) acc[2] += ke; else acc[1] += ke;
      acc[3] += 0.5 * a.w[i] * a.zq[i] * a.phi[k];
      acc[4] += wm * mx;
      acc[5] += wm * my;
      acc[6] += wm * mz;
    }
    if (kd == 0) {
      int zb = a.zq[i];
      zb = zb < 0 ? 0 : (zb >= kHistBins ? kHistBins - 1 : zb);
      hist[zb] += 1;
      histw[zb] += a.w[i];
    }
  }
  DiagPartial* out = a.part + blockIdx.x;
  for (int k = 0; k < 8; ++k) {
    const double s = block_sum<THREADS>(acc[k], red);
    if (threadIdx.x == 0) out->v[k] = s;
  }
  {
    double s = block_sum<THREADS>(static_cast<double>(na), red);
    if (threadIdx.x == 0) out->cnt[0] = static_cast<long long>(s);
    s = block_sum<THREADS>(static_cast<double>(nbad), red);
    if (threadIdx.x == 0) out->cnt[1] = static_cast<long long>(s);
  }
  for (int k = 0; k < kHistBins; ++k) {
    double s = block_sum<THREADS>(static_cast<double>(hist[k]), red);
    if (threadIdx.x == 0) out->hist[k] = static_cast<long long>(s);
    s = block_sum<THREADS>(histw[k], red);
    if (threadIdx.x == 0) out->histw[k] = s;
  }
}

}  // namespace md
