// md_kernels.cu -- instantiations and launchers of the sm_103a kernels.
#include <mutex>

#include "md_device.cuh"
#include "md_internal.h"

namespace md {

// Sums the per-block partials in block order (deterministic); one thread per
// component.
__global__ void k_diag_final(const DiagPartial* __restrict__ part, int nblocks,
                             DiagPartial* __restrict__ out) {
  const int k = threadIdx.x;
  if (k < 8) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b].v[k];
    out->v[k] = s;
  } else if (k < 10) {
    long long s = 0;
    for (int b = 0; b < nblocks; ++b) s += part[b].cnt[k - 8];
    out->cnt[k - 8] = s;
  } else if (k < 10 + kHistBins) {
    long long s = 0;
    for (int b = 0; b < nblocks; ++b) s += part[b].hist[k - 10];
    out->hist[k - 10] = s;
  } else if (k < 10 + 2 * kHistBins) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b].histw[k - 10 - kHistBins];
    out->histw[k - 10 - kHistBins] = s;
  }
}

// ------------------------------------------------------------ layout glue --

// Scatter host-layout records ([n][3] x/u, z, mass, w, kind) into the SoA
// device state of one cluster starting at record `off`; writes the current
// j-stream entry (x, y, z, K_C w z).

// The checks md_set_particles makes of every record, on the staged copy in
// device memory: kind in range, positive mass if active, charge sign matching
// the kind, finite x, u and w.  Records the lowest index that fails.
__global__ void k_validate(const UploadArgs a) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  const unsigned char kd = a.hkind[k];
  const int zq = a.hz[k];
  bool bad = kd > 2;
  bad = bad || (kd != 2 && !(a.hmass[k] > 0.0));
  bad = bad || (kd == 1 && zq >= 0) || (kd == 0 && zq < 0);
  bad = bad || !(isfinite(a.hx[3 * k]) && isfinite(a.hx[3 * k + 1]) && isfinite(a.hx[3 * k + 2]) &&
                 isfinite(a.hu[3 * k]) && isfinite(a.hu[3 * k + 1]) && isfinite(a.hu[3 * k + 2]) &&
                 isfinite(a.hw[k]));
  if (bad) atomicMin(a.first_bad, static_cast<unsigned long long>(k));
}

__global__ void k_upload(const UploadArgs a) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  if (a.first_bad && *a.first_bad != kNoBadRecord) return;  // rejected: state unchanged
  const long long i = a.off + k;
  const unsigned char kd = a.hkind[k];
  const double X = a.hx[3 * k], Y = a.hx[3 * k + 1], Z = a.hx[3 * k + 2];
  a.x[i] = X;
  a.y[i] = Y;
  a.z[i] = Z;
  a.ux[i] = a.hu[3 * k];
  a.uy[i] = a.hu[3 * k + 1];
  a.uz[i] = a.hu[3 * k + 2];
  const int zq = a.hz[k];
  a.zq[i] = zq;
  a.mass[i] = a.hmass[k];
  a.w[i] = a.hw[k];
  a.kind[i] = kd;
  const bool live = (kd != 2);
  a.qm[i] = live ? static_cast<float>(zq / a.hmass[k]) : 0.0f;
  const float q = live ? static_cast<float>(a.kc * a.hw[k] * zq) : 0.0f;
  const float4 p = make_float4(static_cast<float>(X), static_cast<float>(Y), static_cast<float>(Z), q);
  const long long step = __ldcg(a.step);
  if (step & 1) a.posq1[i] = p; else a.posq0[i] = p;
  if (a.vel)
    a.vel[i] = make_float4(static_cast<float>(a.hu[3 * k]), static_cast<float>(a.hu[3 * k + 1]),
                           static_cast<float>(a.hu[3 * k + 2]), static_cast<float>(a.hw[k]));
}

// Energy histogram of the ions (kind ION, z >= 1) of a cluster that the
// detectors have not recorded, at their current u.
__global__ void k_iedf_inside(const ClusterDev c, const double* ux, const double* uy,
                              const double* uz, const double* mass, const int* zq,
                              const unsigned char* kind, const unsigned char* crossed,
                              unsigned long long* hist) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= c.n) return;
  const long long i = c.off + k;
  if (kind[i] != 0 || zq[i] < 1 || crossed[i]) return;
  atomicAdd(hist + det_bin(det_ke_ev(ux[i], uy[i], uz[i], mass[i]), c.det_emax, c.det_nbins),
            1ull);
}

cudaError_t launch_iedf_inside(const ClusterDev& c, const double* ux, const double* uy,
                               const double* uz, const double* mass, const int* zq,
                               const unsigned char* kind, const unsigned char* crossed,
                               unsigned long long* hist, cudaStream_t s) {
  if (c.n <= 0) return cudaSuccess;
  k_iedf_inside<<<static_cast<unsigned>((c.n + 255) / 256), 256, 0, s>>>(c, ux, uy, uz, mass, zq,
                                                                         kind, crossed, hist);
  return cudaGetLastError();
}

// FP64 reference of the direct sum: per target, the plain sum over sources in
// index order of Q_j (x_i - x_j) / (r^2 + eps^2)^{3/2} and Q_j / r, skipping
// the target's own record and uncharged sources, each operation rounded to
// nearest in the order written (no fused multiply-add).  Sources are staged
// through shared memory in tiles of kRefTile.
constexpr int kRefThreads = 128;
constexpr int kRefTile = 256;

__global__ void __launch_bounds__(kRefThreads)
    k_field_fp64(const double* __restrict__ xs, const double* __restrict__ qs, long long ns,
                 const double* __restrict__ xt, const long long* __restrict__ self_idx,
                 long long nt, double eps, double kc, double* e, double* phi) {
  __shared__ double sx[kRefTile], sy[kRefTile], sz[kRefTile], sq[kRefTile];
  const long long i = static_cast<long long>(blockIdx.x) * kRefThreads + threadIdx.x;
  const bool live = i < nt;
  const double xi = live ? xt[3 * i] : 0.0, yi = live ? xt[3 * i + 1] : 0.0,
               zi = live ? xt[3 * i + 2] : 0.0;
  const long long self = (live && self_idx) ? self_idx[i] : -1;
  const double eps2 = __dmul_rn(eps, eps);
  double ex = 0.0, ey = 0.0, ez = 0.0, ph = 0.0;
  for (long long j0 = 0; j0 < ns; j0 += kRefTile) {
    const int cnt = static_cast<int>(ns - j0 < kRefTile ? ns - j0 : kRefTile);
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += kRefThreads) {
      sx[k] = xs[3 * (j0 + k)];
      sy[k] = xs[3 * (j0 + k) + 1];
      sz[k] = xs[3 * (j0 + k) + 2];
      sq[k] = qs[j0 + k];
    }
    __syncthreads();
    if (!live) continue;
    for (int k = 0; k < cnt; ++k) {
      const double q = sq[k];
      if (j0 + k == self || q == 0.0) continue;
      const double dx = __dsub_rn(xi, sx[k]);
      const double dy = __dsub_rn(yi, sy[k]);
      const double dz = __dsub_rn(zi, sz[k]);
      const double r2 = __dadd_rn(
          __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)), eps2);
      const double r = __dsqrt_rn(r2);
      const double inv_r3 = __ddiv_rn(1.0, __dmul_rn(r2, r));
      ex = __dadd_rn(ex, __dmul_rn(__dmul_rn(q, dx), inv_r3));
      ey = __dadd_rn(ey, __dmul_rn(__dmul_rn(q, dy), inv_r3));
      ez = __dadd_rn(ez, __dmul_rn(__dmul_rn(q, dz), inv_r3));
      ph = __dadd_rn(ph, __ddiv_rn(q, r));
    }
  }
  if (!live) return;
  e[3 * i] = __dmul_rn(kc, ex);
  e[3 * i + 1] = __dmul_rn(kc, ey);
  e[3 * i + 2] = __dmul_rn(kc, ez);
  if (phi) phi[i] = __dmul_rn(kc, ph);
}

cudaError_t launch_field_fp64(const double* xs, const double* qs, long long ns, const double* xt,
                              const long long* self_idx, long long nt, double eps, double kc,
                              double* e, double* phi, cudaStream_t s) {
  if (nt <= 0) return cudaSuccess;
  k_field_fp64<<<static_cast<unsigned>((nt + kRefThreads - 1) / kRefThreads), kRefThreads, 0, s>>>(
      xs, qs, ns, xt, self_idx, nt, eps, kc, e, phi);
  return cudaGetLastError();
}

__global__ void k_download(const DownloadArgs a) {  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  const long long i = a.off + k;
  a.hx[3 * k] = a.x[i];
  a.hx[3 * k + 1] = a.y[i];
  a.hx[3 * k + 2] = a.z[i];
  a.hu[3 * k] = a.ux[i];
  a.hu[3 * k + 1] = a.uy[i];
  a.hu[3 * k + 2] = a.uz[i];
  a.hz[k] = a.zq[i];
  a.hmass[k] = a.mass[i];
  a.hw[k] = a.w[i];
  a.hkind[k] = a.kind[i];
}

namespace {

template <int T, int R, int TILE, int ST, bool PK, int MB, bool DET>
cudaError_t launch_step_t(const StepArgs& a, int grid, cudaStream_t s) {
  k_step<T, R, TILE, ST, PK, MB, DET><<<grid, T, 0, s>>>(a);
  return cudaGetLastError();
}

// the diagnostic step (potential summed beside the field)
template <int T, int R, int TILE, int ST, bool PK, int MB>
cudaError_t launch_step_pot_t(const StepArgs& a, int grid, cudaStream_t s) {
  k_step<T, R, TILE, ST, PK, MB, false, true><<<grid, T, 0, s>>>(a);
  return cudaGetLastError();
}

template <int T, int R, int TILE, int ST, bool PK, int MB>
cudaError_t blocks_per_sm_pot_t(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      out, k_step<T, R, TILE, ST, PK, MB, false, true>, T, 0);
}

// minimum-image forces (periodic clusters with min_image)
template <int T, int R, int TILE, int ST, bool PK, int MB>
cudaError_t launch_step_mi_t(const StepArgs& a, int grid, cudaStream_t s) {
  k_step<T, R, TILE, ST, PK, MB, false, false, true><<<grid, T, 0, s>>>(a);
  return cudaGetLastError();
}

template <int T, int R, int TILE, int ST, bool PK, int MB, bool DET = false>
cudaError_t blocks_per_sm_mi_t(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      out, k_step<T, R, TILE, ST, PK, MB, DET, false, true>, T, 0);
}

template <int T, int R, int TILE, int ST, bool PK, int MB>
cudaError_t launch_step_mi_det_t(const StepArgs& a, int grid, cudaStream_t s) {
  k_step<T, R, TILE, ST, PK, MB, true, false, true><<<grid, T, 0, s>>>(a);
  return cudaGetLastError();
}

template <int T, int R, int TILE, int ST, bool PK, int MB, bool DET>
cudaError_t blocks_per_sm_t(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_step<T, R, TILE, ST, PK, MB, DET>,
                                                       T, 0);
}

// threads, i-particles per thread, sources per tile, TMA stages, packed, min CTAs per SM
#define MD_STEP_CONFIG(T, R, TILE, ST, PK, MB)                                          \
  {T, R, TILE, ST, PK, MB, &launch_step_t<T, R, TILE, ST, PK, MB, false>,              \
   &blocks_per_sm_t<T, R, TILE, ST, PK, MB, false>,                                      \
   &launch_step_t<T, R, TILE, ST, PK, MB, true>, &blocks_per_sm_t<T, R, TILE, ST, PK, MB, true>, \
   &launch_step_pot_t<T, R, TILE, ST, PK, MB>, &blocks_per_sm_pot_t<T, R, TILE, ST, PK, MB>,    \
   nullptr, nullptr, nullptr, nullptr}
// ... and with minimum-image forces
#define MD_STEP_CONFIG_MI(T, R, TILE, ST, PK, MB)                                       \
  {T, R, TILE, ST, PK, MB, &launch_step_t<T, R, TILE, ST, PK, MB, false>,              \
   &blocks_per_sm_t<T, R, TILE, ST, PK, MB, false>,                                      \
   &launch_step_t<T, R, TILE, ST, PK, MB, true>, &blocks_per_sm_t<T, R, TILE, ST, PK, MB, true>, \
   &launch_step_pot_t<T, R, TILE, ST, PK, MB>, &blocks_per_sm_pot_t<T, R, TILE, ST, PK, MB>,    \
   &launch_step_mi_t<T, R, TILE, ST, PK, MB>, &blocks_per_sm_mi_t<T, R, TILE, ST, PK, MB>,      \
   &launch_step_mi_det_t<T, R, TILE, ST, PK, MB>,                                        \
   &blocks_per_sm_mi_t<T, R, TILE, ST, PK, MB, true>}
// scalar configurations (all with minimum-image forces)
#define MD_STEP_CONFIG_POT(T, R, TILE, ST, MB)                                          \
  {T, R, TILE, ST, false, MB, &launch_step_t<T, R, TILE, ST, false, MB, false>,          \
   &blocks_per_sm_t<T, R, TILE, ST, false, MB, false>,                                   \
   &launch_step_t<T, R, TILE, ST, false, MB, true>,                                      \
   &blocks_per_sm_t<T, R, TILE, ST, false, MB, true>,                                    \
   &launch_step_pot_t<T, R, TILE, ST, false, MB>, &blocks_per_sm_pot_t<T, R, TILE, ST, false, MB>, \
   &launch_step_mi_t<T, R, TILE, ST, false, MB>, &blocks_per_sm_mi_t<T, R, TILE, ST, false, MB>, \
   &launch_step_mi_det_t<T, R, TILE, ST, false, MB>,                                     \
   &blocks_per_sm_mi_t<T, R, TILE, ST, false, MB, true>}

// min CTAs per SM = 0 leaves the register budget to ptxas; a positive value
// caps it at 64K / (threads x value)
const KernelConfig kConfigs[] = {
    // scalar FP32 pair arithmetic
    MD_STEP_CONFIG_POT(128, 1, 512, 2, 0), MD_STEP_CONFIG_POT(128, 4, 512, 2, 0),
    MD_STEP_CONFIG_POT(256, 2, 512, 2, 0), MD_STEP_CONFIG_POT(128, 8, 512, 2, 0),
    MD_STEP_CONFIG_POT(256, 4, 512, 2, 0),
    // packed f32x2 pair arithmetic (tile expanded in shared memory, one TMA stage)
    MD_STEP_CONFIG(128, 4, 256, 1, true, 0), MD_STEP_CONFIG(256, 4, 256, 1, true, 0),
    MD_STEP_CONFIG_MI(128, 8, 256, 1, true, 0), MD_STEP_CONFIG(128, 4, 512, 1, true, 0),
    MD_STEP_CONFIG_MI(256, 4, 512, 1, true, 0), MD_STEP_CONFIG(128, 8, 512, 1, true, 0),
    // the same with the registers capped for 3 CTAs per SM
    MD_STEP_CONFIG(128, 8, 512, 1, true, 3),
};

// the field kernel: the step kernel's packed source loop (128 threads x 8
// targets, 512-source tiles, one stage)
constexpr int kFieldThreads = 128;
constexpr int kFieldR = 8;
constexpr int kFieldTile = 512;

}  // namespace

const KernelConfig* step_configs(int* count) {
  *count = static_cast<int>(sizeof(kConfigs) / sizeof(kConfigs[0]));
  return kConfigs;
}

// Sum of the segment partials of a split k_field, in segment order, and the
// potential's self term.
__global__ void __launch_bounds__(256) k_field_combine(const FieldArgs a) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.nt) return;
  double ex = 0.0, ey = 0.0, ez = 0.0, ph = 0.0;
  for (int sg = 0; sg < a.nseg; ++sg) {
    const double* p = a.part + 4 * (static_cast<long long>(sg) * a.nt + i);
    ex += p[0];
    ey += p[1];
    ez += p[2];
    ph += p[3];
  }
  a.e[3 * i + 0] = ex;
  a.e[3 * i + 1] = ey;
  a.e[3 * i + 2] = ez;
  if (a.phi) {
    // (a target block without active records has zero partials and stays zero)
    if (a.self_offset >= 0 && ph != 0.0) {
      const long long js = i + a.self_offset;
      if (js < a.ns) ph -= static_cast<double>(a.src[js].w * rsqrt_mufu(a.eps2));
    }
    a.phi[i] = ph;
  }
}

cudaError_t launch_field(const FieldArgs& a, bool potential, cudaStream_t s) {
  if (a.nt <= 0) return cudaSuccess;
  if (a.nseg > 1 && (!a.part || a.seg_len <= 0)) return cudaErrorInvalidValue;
  const long long per = kFieldThreads * kFieldR;
  const dim3 grid(static_cast<unsigned>((a.nt + per - 1) / per),
                  static_cast<unsigned>(a.nseg > 1 ? a.nseg : 1));
  constexpr int T = kFieldThreads, R = kFieldR, TL = kFieldTile;
  if (a.box > 0.0f) {
    if (potential)
      k_field<T, R, TL, 1, true, true, true><<<grid, T, 0, s>>>(a);
    else
      k_field<T, R, TL, 1, false, true, true><<<grid, T, 0, s>>>(a);
  } else if (potential) {
    k_field<T, R, TL, 1, true, false, true><<<grid, T, 0, s>>>(a);
  } else {
    k_field<T, R, TL, 1, false, false, true><<<grid, T, 0, s>>>(a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.nseg <= 1) return e;
  k_field_combine<<<static_cast<unsigned>((a.nt + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

int field_targets_per_cta() { return kFieldThreads * kFieldR; }

cudaError_t field_blocks_per_sm(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      out, k_field<kFieldThreads, kFieldR, kFieldTile, 1, true, false, true>, kFieldThreads, 0);
}

cudaError_t launch_diag(const DiagArgs& a, int blocks, DiagPartial* out, cudaStream_t s) {
  k_diag_partial<kDiagThreads><<<blocks, kDiagThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_diag_final<<<1, 64, 0, s>>>(a.part, blocks, out);
  return cudaGetLastError();
}

// FP32 peak probe: 8 independent FFMA chains per thread, `iters` rounds of 16.
__global__ void __launch_bounds__(256) k_ffma_probe(int iters, float seed, float* sink) {
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = seed + 0.001f * (threadIdx.x + k);
  const float a = 0.9999f, b = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = fmaf(v[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += v[k];
  if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains alive
}

// The same with packed fma.rn.f32x2 (two lanes of FP32 per instruction).
__global__ void __launch_bounds__(256) k_ffma2_probe(int iters, float seed, float* sink) {
  unsigned long long v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float lo = seed + 0.001f * (threadIdx.x + k), hi = lo + 0.5f;
    v[k] = (static_cast<unsigned long long>(__float_as_uint(hi)) << 32) | __float_as_uint(lo);
  }
  const unsigned long long a = (static_cast<unsigned long long>(__float_as_uint(0.9999f)) << 32) |
                               __float_as_uint(0.9999f);
  const unsigned long long b = (static_cast<unsigned long long>(__float_as_uint(1e-7f)) << 32) |
                               __float_as_uint(1e-7f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[k]) : "l"(a), "l"(b));
    }
  }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= v[k];
  if (s == 12345ull) sink[blockIdx.x] = 1.0f;
}

cudaError_t launch_ffma_probe(int blocks, int iters, bool packed, float* sink, cudaStream_t s) {
  if (packed)
    k_ffma2_probe<<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
  else
    k_ffma_probe<<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
  return cudaGetLastError();
}

// Self-test of the bounded waits: one CTA waits on an mbarrier phase that no
// arrival or copy ever completes; the wait gives up after `budget` cycles,
// sets the timeout bit in *err and the kernel returns normally.
__global__ void k_wait_selftest(long long budget, int* err) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (!mbar_wait(&bar, 0u, budget)) {
    if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
  }
}

cudaError_t launch_wait_selftest(long long budget, int* err, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(budget, err);
  return cudaGetLastError();
}

// Records [off, off + n) whose kind is not INACTIVE, added to *out.
__global__ void __launch_bounds__(256) k_count_active(const unsigned char* kind, long long off,
                                                      long long n, unsigned long long* out) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int live = (k < n && kind[off + k] != 2) ? 1 : 0;
  const int cnt = __syncthreads_count(live);
  if (threadIdx.x == 0 && cnt) atomicAdd(out, static_cast<unsigned long long>(cnt));
}

cudaError_t launch_count_active(const unsigned char* kind, long long off, long long n,
                                unsigned long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || n <= 0) return e;
  k_count_active<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(kind, off, n, out);
  return cudaGetLastError();
}

// Records of a generated cluster (Sec. II: atoms at random inside the sphere
// of radius R0; Eq. 1: macro weight w).  Record k is an ion (k < n_ions), an
// electron (k < n_ions + n_electrons) or an inactive slot.
//   Position: uniform in the ball by rejection from the cube [-1, 1]^3.
//     Attempt a draws Philox4x32-10 (key = seed, counter = (k lo, k hi, a,
//     0x67656E01)); s_i = (w_i + 1/2) 2^-31 - 1 (exact), accepted when
//     (s0 s0 + s1 s1) + s2 s2 < 1 with every operation rounded to nearest, so
//     the decision and x = c + r0 s are the same bits as any IEEE FP64
//     evaluation in that order.  64 rejected attempts (2e-21 per record)
//     leave the record at the centre.
//   Momentum: u_i = sigma n_i, Box-Muller normals from the words of counter
//     (k lo, k hi, 0, 0x67656E02): n0, n1 = sqrt(-2 ln v0) (cos, sin)(2 pi v1),
//     n2 = sqrt(-2 ln v2) cos(2 pi v3), v0, v2 = (w + 1) 2^-32,
//     v1, v3 = (w + 1/2) 2^-32.
//   Slots sit at the centre, at rest, z = 0, mass 1.
__global__ void __launch_bounds__(256) k_generate(const GenerateArgs g) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= g.n) return;
  const int kd = k < g.n_ions ? 0 : (k < g.n_ions + g.n_electrons ? 1 : 2);
  const uint2 key = make_uint2(static_cast<uint32_t>(g.seed), static_cast<uint32_t>(g.seed >> 32));
  const uint32_t klo = static_cast<uint32_t>(k), khi = static_cast<uint32_t>(k >> 32);
  double s[3] = {0.0, 0.0, 0.0};
  if (kd != 2) {
    for (uint32_t a = 0; a < 64u; ++a) {
      const uint4 w = philox4x32_10(make_uint4(klo, khi, a, 0x67656E01u), key);
      const double c0 = __dadd_rn(__dmul_rn(__dadd_rn(static_cast<double>(w.x), 0.5), 0x1p-31), -1.0);
      const double c1 = __dadd_rn(__dmul_rn(__dadd_rn(static_cast<double>(w.y), 0.5), 0x1p-31), -1.0);
      const double c2 = __dadd_rn(__dmul_rn(__dadd_rn(static_cast<double>(w.z), 0.5), 0x1p-31), -1.0);
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(c0, c0), __dmul_rn(c1, c1)), __dmul_rn(c2, c2));
      if (r2 < 1.0) {
        s[0] = c0;
        s[1] = c1;
        s[2] = c2;
        break;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) g.x[3 * k + c] = __dadd_rn(g.c[c], __dmul_rn(g.r0, s[c]));
  const double sig = kd == 0 ? g.sig_i : (kd == 1 ? g.sig_e : 0.0);
  double n[3] = {0.0, 0.0, 0.0};
  if (sig > 0.0) {
    const uint4 w = philox4x32_10(make_uint4(klo, khi, 0u, 0x67656E02u), key);
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double v0 = __dmul_rn(__dadd_rn(static_cast<double>(w.x), 1.0), 0x1p-32);
    const double v1 = __dmul_rn(__dadd_rn(static_cast<double>(w.y), 0.5), 0x1p-32);
    const double v2 = __dmul_rn(__dadd_rn(static_cast<double>(w.z), 1.0), 0x1p-32);
    const double v3 = __dmul_rn(__dadd_rn(static_cast<double>(w.w), 0.5), 0x1p-32);
    const double rho = __dsqrt_rn(__dmul_rn(-2.0, log(v0)));
    double sn, cs;
    sincos(__dmul_rn(two_pi, v1), &sn, &cs);
    n[0] = __dmul_rn(rho, cs);
    n[1] = __dmul_rn(rho, sn);
    n[2] = __dmul_rn(__dsqrt_rn(__dmul_rn(-2.0, log(v2))), cos(__dmul_rn(two_pi, v3)));
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) g.u[3 * k + c] = __dmul_rn(sig, n[c]);
  g.kind[k] = static_cast<unsigned char>(kd);
  g.z[k] = kd == 0 ? g.ion_charge : (kd == 1 ? -1 : 0);
  g.mass[k] = kd == 0 ? g.ion_mass : 1.0;
  g.w[k] = g.weight;
}

cudaError_t launch_generate(const GenerateArgs& g, cudaStream_t s) {
  if (g.n <= 0) return cudaSuccess;
  k_generate<<<static_cast<unsigned>((g.n + 255) / 256), 256, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_upload(const UploadArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((a.n + 255) / 256);
  if (a.first_bad) {
    cudaError_t e = cudaMemsetAsync(a.first_bad, 0xff, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_validate<<<grid, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_upload<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_download(const DownloadArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((a.n + 255) / 256);
  k_download<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace md

// ===================================================== allocation-free field
//
// A variant of the field evaluation for callers that cannot allocate device
// memory themselves: code running inside another framework's memory pool, a
// CUDA-graph builder that must not see a cudaMalloc, or a plugin whose host
// forbids allocation after start-up.  Like the split-source step, it cuts the
// sources into segments so that more CTAs share the sum, keeps each segment's
// partial field in scratch memory and lets the last segment to finish add them
// up in segment order.  Here that scratch is a fixed, file-scope device array
// instead of a buffer the library allocates, so the call allocates nothing.
//
// Limits: at most kNoAllocMaxTargets targets per call (sources unbounded), at
// most kNoAllocMaxSeg segments.  The arrays below (about 8.6 MB) are held on
// every GPU that loads the library until the process exits.  Every call shares
// them, so calls that overlap on the GPU (two streams, two host threads) race
// and give wrong fields: serialise them.  Each call clears the counters it
// needs before its kernel runs; the partial sums are overwritten before use.
//
// Both stateless field calls (this one and md_coulomb_field_device) record a
// bounded wait that ran out in one error word per device, also a file-scope
// device array.  The word is sticky: md_field_device_status reads and clears
// it.

namespace md {

constexpr int kNoAllocMaxTargets = 32768;
constexpr int kNoAllocMaxSeg = 8;
constexpr int kNoAllocThreads = 128;
constexpr int kNoAllocR = 2;
constexpr int kNoAllocTile = 512;
constexpr int kNoAllocBlocks = kNoAllocMaxTargets / (kNoAllocThreads * kNoAllocR);

// partial (ex, ey, ez, phi) per segment and target, completion counters per
// target block, and the error word of the stateless field calls (kErrTimeout:
// a bounded wait ran out; kErrBounds: a bounds check of the checked build)
static __device__ __align__(256) double g_noalloc_part[kNoAllocMaxSeg * kNoAllocMaxTargets * 4];
static __device__ __align__(256) unsigned g_noalloc_cnt[kNoAllocBlocks];
static __device__ __align__(256) int g_field_err[1];

struct NoAllocScratch {
  double* part;
  unsigned* cnt;
  int* err;
};

template <int THREADS, int R, int TILE, int STAGES, bool POT>
__global__ void __launch_bounds__(THREADS)
    k_field_noalloc(const FieldArgs a, int nseg, long long seg_len, NoAllocScratch sc) {
  __shared__ Stage<TILE, STAGES> sm;
  __shared__ int s_abort, s_last;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  const int blk = blockIdx.x / nseg;
  const int seg = blockIdx.x % nseg;
  const long long i0 = static_cast<long long>(blk) * (THREADS * R);
  float xi[R], yi[R], zi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = i0 + threadIdx.x + r * THREADS;
    const float4 p = (i < a.nt) ? a.tgt[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
  }
  const long long j0 = static_cast<long long>(seg) * seg_len;
  const long long jrem = a.ns - j0;
  const long long jn = jrem < seg_len ? jrem : seg_len;
  Acc<R, POT> acc;
  acc.zero();
  unsigned it = 0;
  if (!sum_sources<THREADS, R, TILE, STAGES, POT>(sm, it, a.src + j0, jn, xi, yi, zi, a.eps2, acc,
                                                   sc.err, &s_abort))
    return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = i0 + threadIdx.x + r * THREADS;
    if (i >= a.nt) continue;
    double* p = sc.part + 4 * (static_cast<long long>(seg) * kNoAllocMaxTargets + i);
    __stcg(p + 0, -(static_cast<double>(acc.sx[r]) - acc.cx[r]));
    __stcg(p + 1, -(static_cast<double>(acc.sy[r]) - acc.cy[r]));
    __stcg(p + 2, -(static_cast<double>(acc.sz[r]) - acc.cz[r]));
    __stcg(p + 3, POT ? static_cast<double>(acc.sp[r]) - acc.cp[r] : 0.0);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(sc.cnt + blk, 1u);
    s_last = (prev == static_cast<unsigned>(nseg - 1));
    if (s_last) atomicExch(sc.cnt + blk, 0u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = i0 + threadIdx.x + r * THREADS;
    if (i >= a.nt) continue;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int sg = 0; sg < nseg; ++sg) {
      const double* p = sc.part + 4 * (static_cast<long long>(sg) * kNoAllocMaxTargets + i);
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] += __ldcg(p + k);
    }
    a.e[3 * i + 0] = v[0];
    a.e[3 * i + 1] = v[1];
    a.e[3 * i + 2] = v[2];
    if (POT && a.phi) {
      double ph = v[3];
      if (a.self_offset >= 0) {
        const long long js = i + a.self_offset;
        if (js < a.ns) ph -= static_cast<double>(a.src[js].w * rsqrt_mufu(a.eps2));
      }
      a.phi[i] = ph;
    }
  }
}

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
bool g_noalloc_ready[kNoAllocMaxDevices] = {};
NoAllocScratch g_noalloc_ptr[kNoAllocMaxDevices];

// Device addresses of the scratch arrays on the current device, looked up once
// per device (host code cannot use the array names as device addresses).
md_status noalloc_scratch(NoAllocScratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return report_error(MD_ERR_UNSUPPORTED, "device ordinal beyond the allocation-free table");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ready[dev]) {
    NoAllocScratch s;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.part), g_noalloc_part);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaGetSymbolAddress(partials)");
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.cnt), g_noalloc_cnt);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaGetSymbolAddress(counters)");
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.err), g_field_err);
    if (e != cudaSuccess) return report_cuda_error(e, "cudaGetSymbolAddress(error word)");
    g_noalloc_ptr[dev] = s;
    g_noalloc_ready[dev] = true;
  }
  *out = g_noalloc_ptr[dev];
  return MD_OK;
}

}  // namespace

md_status field_error_word(int** out) {
  NoAllocScratch sc;
  const md_status st = noalloc_scratch(&sc);
  if (st == MD_OK) *out = sc.err;
  return st;
}

}  // namespace md

static md_status md_field_device_status_body(void* stream) {
  using namespace md;
  int* word = nullptr;
  md_status st = field_error_word(&word);
  if (st != MD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return report_cuda_error(ce, "cudaStreamSynchronize");
  int v = 0;
  ce = cudaMemcpyAsync(&v, word, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce == cudaSuccess && v != 0) ce = cudaMemsetAsync(word, 0, sizeof(int), s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return report_cuda_error(ce, "reading the field error word");
  if (v & kErrTimeout)
    return report_error(MD_ERR_TIMEOUT,
                        "a stateless field call hit a device-side wait that exceeded its budget; "
                        "its output was not (completely) written");
  if (v & kErrBounds)
    return report_error(MD_ERR_STATE, "a device-side bounds check failed (checked build)");
  return MD_OK;
}

extern "C" md_status md_field_device_status(void* stream) {
  return md::guarded([&] { return md_field_device_status_body(stream); });
}

static md_status md_field_wait_selftest_body(double budget_ms, void* stream) {
  using namespace md;
  if (!(budget_ms > 0.0) || budget_ms > 5000.0)
    return report_error(MD_ERR_ARG, "budget_ms must be in (0, 5000]");
  int* word = nullptr;
  md_status st = field_error_word(&word);
  if (st != MD_OK) return st;
  int dev = 0, clk_khz = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  if (ce != cudaSuccess) return report_cuda_error(ce, "cudaDeviceGetAttribute");
  const long long budget = static_cast<long long>(budget_ms * clk_khz);
  ce = launch_wait_selftest(budget, word, static_cast<cudaStream_t>(stream));
  if (ce != cudaSuccess) return report_cuda_error(ce, "wait self-test launch");
  return MD_OK;
}

extern "C" md_status md_field_wait_selftest(double budget_ms, void* stream) {
  return md::guarded([&] { return md_field_wait_selftest_body(budget_ms, stream); });
}

static md_status md_coulomb_field_device_noalloc_body(const void* src, int64_t ns, const void* tgt,
                                                      int64_t nt, float eps2, int64_t self_offset,
                                                      double* e, double* phi, void* stream) {
  using namespace md;
  if (ns < 0 || nt < 0) return report_error(MD_ERR_ARG, "negative size");
  if (nt > kNoAllocMaxTargets)
    return report_error(MD_ERR_ARG,
                        "md_coulomb_field_device_noalloc: nt exceeds the 32768-target maximum "
                        "of its fixed scratch array");
  if (nt == 0) return MD_OK;
  if (!src || !tgt || !e) return report_error(MD_ERR_ARG, "NULL pointer");
  if ((reinterpret_cast<uintptr_t>(src) & 15) || (reinterpret_cast<uintptr_t>(tgt) & 15))
    return report_error(MD_ERR_ARG, "src and tgt must be 16-byte aligned");
  if (!(eps2 > 0.0f)) return report_error(MD_ERR_ARG, "eps2 must be > 0");
  NoAllocScratch sc;
  md_status st = noalloc_scratch(&sc);
  if (st != MD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long per = kNoAllocThreads * kNoAllocR;
  const int nblk = static_cast<int>((nt + per - 1) / per);
  // segments of at least 4 tiles of sources, at most kNoAllocMaxSeg
  long long nseg = ns / (4LL * kNoAllocTile);
  nseg = nseg < 1 ? 1 : (nseg > kNoAllocMaxSeg ? kNoAllocMaxSeg : nseg);
  const long long seg_len = ns > 0 ? (ns + nseg - 1) / nseg : 1;
  cudaError_t ce = cudaMemsetAsync(sc.cnt, 0, sizeof(unsigned) * nblk, s);
  if (ce != cudaSuccess) return report_cuda_error(ce, "clearing the counters");
  FieldArgs a;
  a.src = static_cast<const float4*>(src);
  a.ns = ns;
  a.tgt = static_cast<const float4*>(tgt);
  a.nt = nt;
  a.eps2 = eps2;
  a.self_offset = self_offset;
  a.e = e;
  a.phi = phi;
  a.err = sc.err;
  a.src_live = nullptr;
  a.tgt_live = nullptr;
  a.gbase = 0;
  const unsigned grid = static_cast<unsigned>(nblk * nseg);
  if (phi)
    k_field_noalloc<kNoAllocThreads, kNoAllocR, kNoAllocTile, 2, true>
        <<<grid, kNoAllocThreads, 0, s>>>(a, static_cast<int>(nseg), seg_len, sc);
  else
    k_field_noalloc<kNoAllocThreads, kNoAllocR, kNoAllocTile, 2, false>
        <<<grid, kNoAllocThreads, 0, s>>>(a, static_cast<int>(nseg), seg_len, sc);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return report_cuda_error(ce, "allocation-free field launch");
  return MD_OK;
}

extern "C" md_status md_coulomb_field_device_noalloc(const void* src, int64_t ns, const void* tgt,
                                                     int64_t nt, float eps2, int64_t self_offset,
                                                     double* e, double* phi, void* stream) {
  return md::guarded([&] { return md_coulomb_field_device_noalloc_body(src, ns, tgt, nt, eps2, self_offset, e, phi, stream); });
}
