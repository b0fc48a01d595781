// md_mlp.cu -- learned surrogate of the ionization rate (not from the paper:
// it stands in for the per-ion rate evaluation nu_ofi + nu_ci of Sec. II).
//
// Network 4 -> 64 -> 64 -> 8 (SiLU hidden layers).  The two hidden layers run
// on the tensor cores with BF16 weights and activations and FP32 accumulation
// (mma.sync.m16n8k16.row.col.f32.bf16.bf16.f32): one warp carries 16 samples
// through both without leaving registers, because the C fragment of an m16n8
// tile (rows g, g+8; columns 2t, 2t+1) is exactly the A fragment slice of the
// next layer's k-step.  The output layer (8 x 64) is a per-sample FP32 dot
// product on the CUDA cores from the FP32 hidden activations, finished by a
// shuffle reduction over the 4 lanes of a quad: BF16 rounding of the last
// layer alone doubles the error of the fitted log-rate, and an ion needs only
// the output row of its own charge state.  At width 64 a layer is a handful of
// mma instructions, so the tcgen05/TMEM machinery would cost more than the
// work it carries.
//
// Features f = ((log10(F/F0) + 1.4)/1.5, z/8, (log10 max(n_e,1e15) - 19.5)/4.5,
//               (log10(max(T_e,0.1)/Ip) + 0.2)/3), F = max(|E|,1e-6) in atomic
// units, Ip the ionization energy of charge state z, F0 = (2 Ip/E_h)^(3/2);
// output y_k ~ (log10(nu_k + 1e-12) + 6)/6 for z = k -> k+1, inverted as
// nu = max(10^(6y - 6) - 1e-12, 0): rates below 1e-12 per unit time (P < 1e-13
// per pass) never ionize, and the additive floor keeps the target smooth.
// Parameters (FP32 master copy): W1[64][4] b1[64] W2[64][64] b2[64] W3[8][64] b3[8].
//
// Training: samples (|E|, z, n_e, T_e) drawn log-uniformly by Philox and
// labelled by the library's own FP64 plain rate; minibatch forward/backward
// (hidden-layer activation gradients on the tensor cores, weight gradients
// accumulated per CTA in FP32 in a fixed order), then a deterministic
// reduction and Adam.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "md_device.cuh"
#include "md_internal.h"

namespace md {

namespace {

constexpr int kNI = 4, kNH = 64, kNO = 8;
constexpr int kOffW1 = 0, kOffB1 = 256, kOffW2 = 320, kOffB2 = 4416, kOffW3 = 4480, kOffB3 = 4992;
constexpr int kNParam = 5000;
constexpr int kWarps = 4;                 // warps per CTA, 16 samples each
constexpr int kTileSamples = 16 * kWarps; // samples per CTA iteration

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_round(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu(float a) { return a / (1.0f + __expf(-a)); }

// Element o of an 8-vector held in registers, without dynamic indexing
// (which would move the whole fragment state to local memory).
__device__ __forceinline__ float pick8(const float (&v)[8], int o) {
  float r = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) r = (k == o) ? v[k] : r;
  return r;
}

__device__ __forceinline__ float dsilu(float a) {
  const float s = 1.0f / (1.0f + __expf(-a));
  return s * (1.0f + a * (1.0f - s));
}

// Weights of one CTA in shared memory: BF16 hidden-layer matrices (W1 padded
// to K = 16), FP32 output layer and biases.
struct MlpWeights {
  alignas(16) __nv_bfloat16 w1[kNH][16];
  alignas(16) __nv_bfloat16 w2[kNH][kNH];
  alignas(16) float w3[kNO][kNH];
  float b1[kNH], b2[kNH], b3[kNO];
};

__device__ void load_weights(const float* __restrict__ p, MlpWeights& w) {
  for (int e = threadIdx.x; e < kNH * 16; e += blockDim.x) {
    const int n = e >> 4, k = e & 15;
    w.w1[n][k] = __float2bfloat16_rn(k < kNI ? p[kOffW1 + n * kNI + k] : 0.0f);
  }
  for (int e = threadIdx.x; e < kNH * kNH; e += blockDim.x)
    w.w2[e >> 6][e & 63] = __float2bfloat16_rn(p[kOffW2 + e]);
  for (int e = threadIdx.x; e < kNO * kNH; e += blockDim.x)
    w.w3[e >> 6][e & 63] = p[kOffW3 + e];
  for (int e = threadIdx.x; e < kNH; e += blockDim.x) {
    w.b1[e] = p[kOffB1 + e];
    w.b2[e] = p[kOffB2 + e];
  }
  for (int e = threadIdx.x; e < kNO; e += blockDim.x) w.b3[e] = p[kOffB3 + e];
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ uint32_t pair_of(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
         (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
}

// Forward state of one warp's 16 samples (fragments; lane = 4 g + t).
struct Fwd {
  float a1[8][4];     // layer-1 pre-activations, C layout per n-tile
  float a2[8][4];     // layer-2 pre-activations
  uint32_t h1[4][4];  // silu(a1) as BF16 A fragments of layer 2 (per k-step)
  float yall[2][kNO]; // all outputs of rows g and g+8 (every lane of the quad)
  float y[4];         // outputs: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)
};

// C tiles (8 n-tiles of 16x8, FP32) -> activation -> A fragments of 4 k-steps.
__device__ __forceinline__ void c_to_a(const float (&c)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a[kk][0] = pack_bf16(silu(c[2 * kk][0]), silu(c[2 * kk][1]));
    a[kk][1] = pack_bf16(silu(c[2 * kk][2]), silu(c[2 * kk][3]));
    a[kk][2] = pack_bf16(silu(c[2 * kk + 1][0]), silu(c[2 * kk + 1][1]));
    a[kk][3] = pack_bf16(silu(c[2 * kk + 1][2]), silu(c[2 * kk + 1][3]));
  }
}

// x: features of rows g and g+8 of this warp's tile (x_lo, x_hi: 4 values).
// Hidden layers only: a1, h1, a2.
__device__ __forceinline__ void forward_hidden(const MlpWeights& w, const float (&xg)[4],
                                               const float (&xg8)[4], Fwd& f) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // layer 1: A = features padded to K = 16 (columns 0..3 real)
  const uint32_t x0 = t < 2 ? pack_bf16(xg[2 * t], xg[2 * t + 1]) : 0u;
  const uint32_t x1 = t < 2 ? pack_bf16(xg8[2 * t], xg8[2 * t + 1]) : 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = w.b1[8 * j + 2 * t], b1 = w.b1[8 * j + 2 * t + 1];
    f.a1[j][0] = b0; f.a1[j][1] = b1; f.a1[j][2] = b0; f.a1[j][3] = b1;
    mma_bf16(f.a1[j], x0, x1, 0u, 0u, ld_pair(&w.w1[8 * j + g][2 * t]), 0u);
  }
  c_to_a(f.a1, f.h1);
  // layer 2
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float b0 = w.b2[8 * j + 2 * t], b1 = w.b2[8 * j + 2 * t + 1];
    f.a2[j][0] = b0; f.a2[j][1] = b1; f.a2[j][2] = b0; f.a2[j][3] = b1;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(f.a2[j], f.h1[kk][0], f.h1[kk][1], f.h1[kk][2], f.h1[kk][3],
               ld_pair(&w.w2[8 * j + g][16 * kk + 2 * t]),
               ld_pair(&w.w2[8 * j + g][16 * kk + 8 + 2 * t]));
  }
}

// All 8 outputs of rows g and g+8 (every lane of the quad gets them).
__device__ __forceinline__ void forward(const MlpWeights& w, const float (&xg)[4],
                                        const float (&xg8)[4], Fwd& f) {
  forward_hidden(w, xg, xg8, f);
  const int t = threadIdx.x & 3;
  // layer 3 in FP32: partial dot products over this lane's 16 columns of
  // rows g and g+8, summed over the quad (lanes t = 0..3)
#pragma unroll
  for (int o = 0; o < kNO; ++o) {
    float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float w0 = w.w3[o][8 * j + 2 * t], w1 = w.w3[o][8 * j + 2 * t + 1];
      p0 = fmaf(w0, silu(f.a2[j][0]), fmaf(w1, silu(f.a2[j][1]), p0));
      p1 = fmaf(w0, silu(f.a2[j][2]), fmaf(w1, silu(f.a2[j][3]), p1));
    }
    p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
    p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
    p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
    f.yall[0][o] = p0 + w.b3[o];
    f.yall[1][o] = p1 + w.b3[o];
  }
#pragma unroll
  for (int o = 0; o < kNO; ++o) {
    if (o == 2 * t) { f.y[0] = f.yall[0][o]; f.y[2] = f.yall[1][o]; }
    if (o == 2 * t + 1) { f.y[1] = f.yall[0][o]; f.y[3] = f.yall[1][o]; }
  }
}

// Surrogate inputs of an ion of charge z: field relative to the tunnelling
// scale F0 = (2 Ip/E_h)^(3/2) of that charge state (atomic units), density,
// temperature relative to Ip.  FP32 (the first layer rounds them to BF16).
__device__ __forceinline__ void features_of(const IonDev& io, double emag, int z, double ne,
                                            double te, float* f) {
  const float ip = static_cast<float>(io.ip_ev[z]);
  const float fau = static_cast<float>(rate::kMeC2Ev * io.k_si / rate::kFieldAu);
  const float lf = log10f(fmaxf(static_cast<float>(emag), 1e-6f)) + log10f(fau);
  const float lf0 = 1.5f * log10f(2.0f * ip / static_cast<float>(rate::kHartreeEv));
  f[0] = (lf - lf0 + 1.4f) / 1.5f;
  f[1] = static_cast<float>(z) / 8.0f;
  f[2] = (log10f(fmaxf(static_cast<float>(ne), 1e15f)) - 19.5f) / 4.5f;
  f[3] = (log10f(fmaxf(static_cast<float>(te), 0.1f) / ip) + 0.2f) / 3.0f;
}

// Rate from the network output: nu = max(10^(6y - 6) - 1e-12, 0), the power
// in FP32 (the surrogate is good to a few per cent), the floor in FP64.
__device__ __forceinline__ double rate_of_output(float y) {
  return fmax(static_cast<double>(exp10f(6.0f * y - 6.0f)) - 1e-12, 0.0);
}

// Output of the charge state of each row only (rows g and g+8 of the warp's
// tile): the FP32 dot product of that row of W3, summed over the quad.
__device__ __forceinline__ void forward_sel(const MlpWeights& w, const float (&xg)[4],
                                            const float (&xg8)[4], int z0, int z1,
                                            float (&ysel)[2]) {
  Fwd f;
  forward_hidden(w, xg, xg8, f);
  const int t = threadIdx.x & 3;
  float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c0 = 8 * j + 2 * t;
    p0 = fmaf(w.w3[z0][c0], silu(f.a2[j][0]), fmaf(w.w3[z0][c0 + 1], silu(f.a2[j][1]), p0));
    p1 = fmaf(w.w3[z1][c0], silu(f.a2[j][2]), fmaf(w.w3[z1][c0 + 1], silu(f.a2[j][3]), p1));
  }
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  ysel[0] = p0 + w.b3[z0];
  ysel[1] = p1 + w.b3[z1];
}

// ------------------------------------------------------------ inference --

__global__ void __launch_bounds__(32 * kWarps) k_mlp_forward(const float* __restrict__ p,
                                                             const float* __restrict__ feats,
                                                             long long n, float* __restrict__ y) {
  __shared__ MlpWeights w;
  load_weights(p, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long tiles = (n + 15) / 16;
  for (long long tile = static_cast<long long>(blockIdx.x) * kWarps + (threadIdx.x >> 5);
       tile < tiles; tile += static_cast<long long>(gridDim.x) * kWarps) {
    const long long s0 = tile * 16 + g, s1 = s0 + 8;
    float xg[4], xg8[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xg[k] = s0 < n ? feats[4 * s0 + k] : 0.0f;
      xg8[k] = s1 < n ? feats[4 * s1 + k] : 0.0f;
    }
    Fwd f;
    forward(w, xg, xg8, f);
    if (s0 < n) { y[8 * s0 + 2 * t] = f.y[0]; y[8 * s0 + 2 * t + 1] = f.y[1]; }
    if (s1 < n) { y[8 * s1 + 2 * t] = f.y[2]; y[8 * s1 + 2 * t + 1] = f.y[3]; }
  }
}

// Ionization pass, rate_model 2: for every ion inside the training domain
// the surrogate rate nu = 10^(15 y_z - 15); ions outside keep use_plain = 1.
__global__ void __launch_bounds__(32 * kWarps) k_ion_mlp_rates(const IonArgs a) {
  __shared__ MlpWeights w;
  const long long step = __ldcg(a.step);
  if (a.ion.rate_model != 2) return;
  if (!a.force && !(a.ion.ionize_every > 0 && step % a.ion.ionize_every == 0)) return;
  load_weights(a.mlp, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long n = a.ion.n_ions;
  const long long tiles = (n + 15) / 16;
  for (long long tile = static_cast<long long>(blockIdx.x) * kWarps + (threadIdx.x >> 5);
       tile < tiles; tile += static_cast<long long>(gridDim.x) * kWarps) {
    const long long s[2] = {tile * 16 + g, tile * 16 + g + 8};
    float x[2][4];
    int zs[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      zs[h] = -1;
      x[h][0] = x[h][1] = x[h][2] = x[h][3] = 0.0f;
      if (s[h] < n) {
        const double* o = a.out + 4 * s[h];
        zs[h] = a.zq[a.c.off + s[h]];
        features_of(a.ion, o[0], zs[h] < 0 ? 0 : (zs[h] < kNO ? zs[h] : kNO - 1), o[1], o[2],
                    x[h]);
      }
    }
    float ysel[2];
    forward_sel(w, x[0], x[1], zs[0] < 0 ? 0 : (zs[0] < kNO ? zs[0] : kNO - 1),
                zs[1] < 0 ? 0 : (zs[1] < kNO ? zs[1] : kNO - 1), ysel);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (t != 0 || s[h] >= n || zs[h] < 0 || zs[h] >= a.ion.zmax) continue;
      const double* o = a.out + 4 * s[h];
      const bool inside = o[0] >= a.ion.dom[0] && o[0] <= a.ion.dom[1] &&
                          (o[1] == 0.0 || (o[1] >= a.ion.dom[2] && o[1] <= a.ion.dom[3])) &&
                          (o[1] == 0.0 || (o[2] >= a.ion.dom[4] && o[2] <= a.ion.dom[5]));
      if (!inside) continue;
      a.nu[s[h]] = rate_of_output(ysel[h]);
    }
  }
}

// -------------------------------------------------------------- training --

// Per-warp staging for the weight gradients: x and h1 (BF16-rounded, as the
// tensor-core layers use them), h2 (FP32), dy, da1, da2 of 16 samples.
struct WarpStage {
  float x[16][kNI];
  float h1[16][kNH];
  float h2[16][kNH];
  float dy[16][kNO];
  float da1[16][kNH];
  float da2[16][kNH];
};

struct TrainSmem {
  MlpWeights w;
  WarpStage st[kWarps];
  float loss[kWarps];
};

// One minibatch [b0, b0 + nb) of the sample set: forward, backward, per-CTA
// FP32 gradient partials (fixed accumulation order) and loss partials.
__global__ void __launch_bounds__(32 * kWarps) k_mlp_train(const float* __restrict__ p,
                                                           const float* __restrict__ feats,
                                                           const int* __restrict__ zs,
                                                           const float* __restrict__ target,
                                                           long long b0, long long nb,
                                                           float* __restrict__ part,
                                                           float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  load_weights(p, S.w);
  __syncthreads();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const float coef = 2.0f / static_cast<float>(nb);
  // owned gradient entries
  float gw2[32], gw3[4], gw1[2], gb = 0.0f, gb3 = 0.0f;
#pragma unroll
  for (int m = 0; m < 32; ++m) gw2[m] = 0.0f;
#pragma unroll
  for (int m = 0; m < 4; ++m) gw3[m] = 0.0f;
  gw1[0] = gw1[1] = 0.0f;
  float lsum = 0.0f;
  const int kcol = tid & 63, nrow = tid >> 6;
  const long long iters = (nb + kTileSamples - 1) / kTileSamples;
  for (long long it = blockIdx.x; it < iters; it += gridDim.x) {
    WarpStage& st = S.st[warp];
    const long long base = b0 + it * kTileSamples + warp * 16;
    const long long lim = b0 + nb;
    const long long sg = base + g, sg8 = base + g + 8;
    float xg[4], xg8[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xg[k] = sg < lim ? feats[4 * sg + k] : 0.0f;
      xg8[k] = sg8 < lim ? feats[4 * sg8 + k] : 0.0f;
    }
    Fwd f;
    forward(S.w, xg, xg8, f);
    // dL/dy: only the output of the sample's charge state
    const int zg = sg < lim ? zs[sg] : -1, zg8 = sg8 < lim ? zs[sg8] : -1;
    const float tg = sg < lim ? target[sg] : 0.0f, tg8 = sg8 < lim ? target[sg8] : 0.0f;
    float dy[4];
    dy[0] = (zg == 2 * t) ? coef * (f.y[0] - tg) : 0.0f;
    dy[1] = (zg == 2 * t + 1) ? coef * (f.y[1] - tg) : 0.0f;
    dy[2] = (zg8 == 2 * t) ? coef * (f.y[2] - tg8) : 0.0f;
    dy[3] = (zg8 == 2 * t + 1) ? coef * (f.y[3] - tg8) : 0.0f;
    if (zg == 2 * t) lsum += (f.y[0] - tg) * (f.y[0] - tg);
    if (zg == 2 * t + 1) lsum += (f.y[1] - tg) * (f.y[1] - tg);
    if (zg8 == 2 * t) lsum += (f.y[2] - tg8) * (f.y[2] - tg8);
    if (zg8 == 2 * t + 1) lsum += (f.y[3] - tg8) * (f.y[3] - tg8);
    // dh2 = dy W3 in FP32: every lane of the quad has both rows' outputs, so
    // each forms the gradient of its own 16 columns from the selected row of W3
    const float dsel0 = (zg >= 0 && zg < kNO) ? coef * (pick8(f.yall[0], zg) - tg) : 0.0f;
    const float dsel1 = (zg8 >= 0 && zg8 < kNO) ? coef * (pick8(f.yall[1], zg8) - tg8) : 0.0f;
    const int zr0 = (zg >= 0 && zg < kNO) ? zg : 0, zr1 = (zg8 >= 0 && zg8 < kNO) ? zg8 : 0;
    float dh[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c0 = 8 * j + 2 * t;
      dh[j][0] = dsel0 * S.w.w3[zr0][c0];
      dh[j][1] = dsel0 * S.w.w3[zr0][c0 + 1];
      dh[j][2] = dsel1 * S.w.w3[zr1][c0];
      dh[j][3] = dsel1 * S.w.w3[zr1][c0 + 1];
    }
    // da2 = dh2 * silu'(a2); stage h2 (FP32, as the output layer uses it), h1
    // (BF16, as layer 2 uses it), dy, da2
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int q = 0; q < 4; ++q) dh[j][q] *= dsilu(f.a2[j][q]);
      const int c0 = 8 * j + 2 * t;
      st.da2[g][c0] = dh[j][0]; st.da2[g][c0 + 1] = dh[j][1];
      st.da2[g + 8][c0] = dh[j][2]; st.da2[g + 8][c0 + 1] = dh[j][3];
      st.h2[g][c0] = silu(f.a2[j][0]);
      st.h2[g][c0 + 1] = silu(f.a2[j][1]);
      st.h2[g + 8][c0] = silu(f.a2[j][2]);
      st.h2[g + 8][c0 + 1] = silu(f.a2[j][3]);
      st.h1[g][c0] = bf16_round(silu(f.a1[j][0]));
      st.h1[g][c0 + 1] = bf16_round(silu(f.a1[j][1]));
      st.h1[g + 8][c0] = bf16_round(silu(f.a1[j][2]));
      st.h1[g + 8][c0 + 1] = bf16_round(silu(f.a1[j][3]));
    }
    st.dy[g][2 * t] = dy[0]; st.dy[g][2 * t + 1] = dy[1];
    st.dy[g + 8][2 * t] = dy[2]; st.dy[g + 8][2 * t + 1] = dy[3];
    // dh1 = da2 W2 (A = da2 as BF16 fragments)
    uint32_t da[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      da[kk][0] = pack_bf16(dh[2 * kk][0], dh[2 * kk][1]);
      da[kk][1] = pack_bf16(dh[2 * kk][2], dh[2 * kk][3]);
      da[kk][2] = pack_bf16(dh[2 * kk + 1][0], dh[2 * kk + 1][1]);
      da[kk][3] = pack_bf16(dh[2 * kk + 1][2], dh[2 * kk + 1][3]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float d1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t bb0 = pair_of(S.w.w2[16 * kk + 2 * t][8 * j + g],
                                     S.w.w2[16 * kk + 2 * t + 1][8 * j + g]);
        const uint32_t bb1 = pair_of(S.w.w2[16 * kk + 8 + 2 * t][8 * j + g],
                                     S.w.w2[16 * kk + 9 + 2 * t][8 * j + g]);
        mma_bf16(d1, da[kk][0], da[kk][1], da[kk][2], da[kk][3], bb0, bb1);
      }
      const int c0 = 8 * j + 2 * t;
      st.da1[g][c0] = d1[0] * dsilu(f.a1[j][0]);
      st.da1[g][c0 + 1] = d1[1] * dsilu(f.a1[j][1]);
      st.da1[g + 8][c0] = d1[2] * dsilu(f.a1[j][2]);
      st.da1[g + 8][c0 + 1] = d1[3] * dsilu(f.a1[j][3]);
    }
    if (t == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        st.x[g][k] = bf16_round(xg[k]);
        st.x[g + 8][k] = bf16_round(xg8[k]);
      }
    }
    __syncthreads();
    // weight gradients of the CTA's 64 samples, in sample order
    for (int wv = 0; wv < kWarps; ++wv) {
      const WarpStage& sw = S.st[wv];
      for (int s = 0; s < 16; ++s) {
        const float h1k = sw.h1[s][kcol], h2k = sw.h2[s][kcol];
#pragma unroll
        for (int m = 0; m < 32; ++m) gw2[m] = fmaf(sw.da2[s][nrow + 2 * m], h1k, gw2[m]);
#pragma unroll
        for (int m = 0; m < 4; ++m) gw3[m] = fmaf(sw.dy[s][nrow + 2 * m], h2k, gw3[m]);
        const float xk = sw.x[s][tid & 3];
        gw1[0] = fmaf(sw.da1[s][tid >> 2], xk, gw1[0]);
        gw1[1] = fmaf(sw.da1[s][(tid >> 2) + 32], xk, gw1[1]);
        gb += (tid < 64) ? sw.da1[s][tid] : sw.da2[s][tid - 64];
        if (tid < kNO) gb3 += sw.dy[s][tid];
      }
    }
    __syncthreads();
  }
  // per-CTA partials: [blockIdx][kNParam]
  float* out = part + static_cast<long long>(blockIdx.x) * kNParam;
#pragma unroll
  for (int m = 0; m < 32; ++m) out[kOffW2 + (nrow + 2 * m) * kNH + kcol] = gw2[m];
#pragma unroll
  for (int m = 0; m < 4; ++m) out[kOffW3 + (nrow + 2 * m) * kNH + kcol] = gw3[m];
  out[kOffW1 + (tid >> 2) * kNI + (tid & 3)] = gw1[0];
  out[kOffW1 + ((tid >> 2) + 32) * kNI + (tid & 3)] = gw1[1];
  if (tid < 64) out[kOffB1 + tid] = gb; else out[kOffB2 + tid - 64] = gb;
  if (tid < kNO) out[kOffB3 + tid] = gb3;
  // loss partial: lanes hold disjoint samples, summed in lane then warp order
  float l = lsum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if (lane == 0) S.loss[warp] = l;
  __syncthreads();
  if (tid == 0) {
    float tot = 0.0f;
    for (int k = 0; k < kWarps; ++k) tot += S.loss[k];
    loss_part[blockIdx.x] = tot;
  }
}

// Training samples: |E|, n_e, T_e log-uniform over the domain, z uniform in
// [0, zmax); label = target of the library's FP64 plain rate.  Philox keyed
// on the seed, counter (sample, 0x5A3D0001, 0, 0).
__global__ void k_mlp_samples(IonDev io, long long n, unsigned long long seed, float* feats,
                              int* zs, float* target, double* raw) {
  const long long s = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint4 w = philox4x32_10(
      make_uint4(static_cast<uint32_t>(s), 0x5A3D0001u, static_cast<uint32_t>(s >> 32), 0u),
      make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
  const double u0 = (w.x + 0.5) * (1.0 / 4294967296.0);
  const double u2 = (w.z + 0.5) * (1.0 / 4294967296.0);
  const double u3 = (w.w + 0.5) * (1.0 / 4294967296.0);
  const double le = log10(io.dom[0]) + u0 * (log10(io.dom[1]) - log10(io.dom[0]));
  const double ln = log10(io.dom[2]) + u2 * (log10(io.dom[3]) - log10(io.dom[2]));
  const double lt = log10(io.dom[4]) + u3 * (log10(io.dom[5]) - log10(io.dom[4]));
  const double emag = pow(10.0, le), ne = pow(10.0, ln), te = pow(10.0, lt);
  const int z = static_cast<int>(w.y % static_cast<uint32_t>(io.zmax));
  const double nu = rate::rate_plain(io, emag, z, ne, te);
  features_of(io, emag, z, ne, te, feats + 4 * s);
  zs[s] = z;
  target[s] = static_cast<float>((log10(fmax(nu, 0.0) + 1e-12) + 6.0) / 6.0);
  if (raw) {
    raw[3 * s] = emag;
    raw[3 * s + 1] = ne;
    raw[3 * s + 2] = te;
  }
}

// Uniform(-a, a) weights with a = sqrt(6 / (fan_in + fan_out)), zero biases.
__global__ void k_mlp_init(float* p, unsigned long long seed) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNParam) return;
  double a = 0.0;
  if (e < kOffB1) a = sqrt(6.0 / (kNI + kNH));
  else if (e >= kOffW2 && e < kOffB2) a = sqrt(6.0 / (kNH + kNH));
  else if (e >= kOffW3 && e < kOffB3) a = sqrt(6.0 / (kNH + kNO));
  const uint4 w = philox4x32_10(make_uint4(static_cast<uint32_t>(e), 0x5A3D0002u, 0u, 0u),
                                make_uint2(static_cast<uint32_t>(seed),
                                           static_cast<uint32_t>(seed >> 32)));
  const double u = (w.x + 0.5) * (1.0 / 4294967296.0);
  p[e] = static_cast<float>(a * (2.0 * u - 1.0));
}

// Sum of the per-CTA gradient partials in CTA order, then one Adam step.
__global__ void k_mlp_adam(float* p, float* m, float* v, const float* part, int nparts,
                           float lr, float b1, float b2, float eps, int step, float* grad_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNParam) return;
  float g = 0.0f;
  for (int k = 0; k < nparts; ++k) g += part[static_cast<long long>(k) * kNParam + e];
  if (grad_out) grad_out[e] = g;
  if (lr <= 0.0f) return;
  const float mk = b1 * m[e] + (1.0f - b1) * g;
  const float vk = b2 * v[e] + (1.0f - b2) * g * g;
  m[e] = mk;
  v[e] = vk;
  const float mh = mk / (1.0f - powf(b1, static_cast<float>(step)));
  const float vh = vk / (1.0f - powf(b2, static_cast<float>(step)));
  p[e] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_sum_floats(const float* x, int n, float* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float s = 0.0f;
  for (int k = 0; k < n; ++k) s += x[k];
  *out = s;
}

// Rates of independent ions: surrogate inside the domain (model 2), -1 else.
__global__ void __launch_bounds__(32 * kWarps) k_rates_mlp(IonDev io, const float* __restrict__ p,
                                                           const double* emag, const int* zs,
                                                           const double* ne, const double* te,
                                                           long long n, double* nu) {
  __shared__ MlpWeights w;
  load_weights(p, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long tiles = (n + 15) / 16;
  for (long long tile = static_cast<long long>(blockIdx.x) * kWarps + (threadIdx.x >> 5);
       tile < tiles; tile += static_cast<long long>(gridDim.x) * kWarps) {
    const long long s[2] = {tile * 16 + g, tile * 16 + g + 8};
    float x[2][4];
    int z[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      z[h] = s[h] < n ? zs[s[h]] : 0;
      x[h][0] = x[h][1] = x[h][2] = x[h][3] = 0.0f;
      if (s[h] < n)  // out-of-range charges get a valid row here and no surrogate rate below
        features_of(io, emag[s[h]], z[h] < 0 ? 0 : (z[h] < kNO ? z[h] : kNO - 1), ne[s[h]],
                    te[s[h]], x[h]);
    }
    float ysel[2];
    forward_sel(w, x[0], x[1], z[0] < 0 ? 0 : (z[0] < kNO ? z[0] : kNO - 1),
                z[1] < 0 ? 0 : (z[1] < kNO ? z[1] : kNO - 1), ysel);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (t != 0 || s[h] >= n) continue;  // lane t = 0 of the quad writes
      const long long k = s[h];
      const bool inside = z[h] >= 0 && z[h] < io.zmax && emag[k] >= io.dom[0] &&
                          emag[k] <= io.dom[1] &&
                          (ne[k] == 0.0 || (ne[k] >= io.dom[2] && ne[k] <= io.dom[3] &&
                                            te[k] >= io.dom[4] && te[k] <= io.dom[5]));
      nu[k] = inside ? rate_of_output(ysel[h]) : -1.0;
    }
  }
}

// Plain rates where no surrogate rate was set (all of them when fill_all).
__global__ void k_rates_plain(IonDev io, const double* emag, const int* zs, const double* ne,
                              const double* te, long long n, double* nu, int fill_all) {
  const long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  if (!fill_all && nu[k] >= 0.0) return;
  const int z = zs[k];
  nu[k] = (z >= 0 && z < io.zmax) ? rate::rate_plain(io, emag[k], z, ne[k], te[k]) : 0.0;
}

int train_grid() {
  static int g = 0;
  if (!g) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g = 2 * (sms > 0 ? sms : 1);
  }
  return g;
}

cudaError_t train_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sizeof(TrainSmem)));
  if (e == cudaSuccess) done = true;
  return e;
}

IonDev domain_io(const md_mlp_train_config& c) {
  IonDev io;
  std::memset(&io, 0, sizeof(io));
  io.zmax = c.zmax;
  io.k_si = 2.0 * 3.14159265358979323846 / (c.lambda_um * 1e-6);
  io.omega = 299792458.0 * io.k_si;
  for (int z = 0; z < kMaxZ; ++z) {
    io.ip_ev[z] = c.ip_ev[z];
    io.q_outer[z] = c.q_outer[z];
  }
  io.dom[0] = c.e_min; io.dom[1] = c.e_max;
  io.dom[2] = c.ne_min; io.dom[3] = c.ne_max;
  io.dom[4] = c.te_min; io.dom[5] = c.te_max;
  return io;
}

md_status check_train_config(const md_mlp_train_config* c) {
  if (!c) return report_error(MD_ERR_ARG, "NULL training configuration");
  if (c->zmax < 1 || c->zmax > kNO)
    return report_error(MD_ERR_ARG, "surrogate zmax must be in [1, 8] (8 outputs)");
  if (!(c->lambda_um > 0.0)) return report_error(MD_ERR_ARG, "lambda_um must be > 0");
  if (!(c->e_min > 0.0 && c->e_max > c->e_min && c->ne_min > 0.0 && c->ne_max > c->ne_min &&
        c->te_min > 0.0 && c->te_max > c->te_min))
    return report_error(MD_ERR_ARG, "bad surrogate domain");
  for (int z = 0; z < c->zmax; ++z)
    if (!(c->ip_ev[z] > 0.0)) return report_error(MD_ERR_ARG, "ip_ev must be > 0 below zmax");
  return MD_OK;
}

}  // namespace

cudaError_t launch_ion_mlp(const IonArgs& a, cudaStream_t s) {
  if (!a.mlp) return cudaErrorInvalidValue;
  const long long tiles = (a.ion.n_ions + 15) / 16;
  const unsigned grid = static_cast<unsigned>((tiles + kWarps - 1) / kWarps);
  k_ion_mlp_rates<<<grid, 32 * kWarps, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace md

using md::report_cuda_error;
using md::report_error;

#define MLP_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return report_cuda_error(e_, #call);     \
  } while (0)

extern "C" {

static md_status md_mlp_forward_device_body(const float* params, const float* feats, int64_t n, float* y,
                                            void* stream) {
  if (n < 0) return report_error(MD_ERR_ARG, "n < 0");
  if (n == 0) return MD_OK;
  if (!params || !feats || !y) return report_error(MD_ERR_ARG, "NULL pointer");
  const long long tiles = (n + 15) / 16;
  const unsigned grid = static_cast<unsigned>(
      std::min<long long>((tiles + md::kWarps - 1) / md::kWarps, 4096));
  md::k_mlp_forward<<<grid, 32 * md::kWarps, 0, static_cast<cudaStream_t>(stream)>>>(params, feats,
                                                                                   n, y);
  MLP_CUDA(cudaGetLastError());
  return MD_OK;
}

md_status md_mlp_forward_device(const float* params, const float* feats, int64_t n, float* y,
                                void* stream) {
  return md::guarded([&] { return md_mlp_forward_device_body(params, feats, n, y, stream); });
}

static md_status md_mlp_loss_grad_device_body(const float* params, const float* feats, const int32_t* z,
                                              const float* target, int64_t n, float* grad, float* loss,
                                              void* stream) {
  if (n <= 0) return report_error(MD_ERR_ARG, "n must be > 0");
  if (!params || !feats || !z || !target || !grad) return report_error(MD_ERR_ARG, "NULL pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MLP_CUDA(md::train_smem_attr());
  const int grid = md::train_grid();
  float* part = nullptr;
  float* lpart = nullptr;
  MLP_CUDA(cudaMalloc(reinterpret_cast<void**>(&part), sizeof(float) * grid * md::kNParam));
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&lpart), sizeof(float) * grid);
  if (e == cudaSuccess) {
    md::k_mlp_train<<<grid, 32 * md::kWarps, sizeof(md::TrainSmem), s>>>(params, feats, z, target,
                                                                         0, n, part, lpart);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    md::k_mlp_adam<<<(md::kNParam + 255) / 256, 256, 0, s>>>(nullptr, nullptr, nullptr, part, grid,
                                                            0.0f, 0.f, 0.f, 0.f, 1, grad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && loss) {
    md::k_sum_floats<<<1, 1, 0, s>>>(lpart, grid, loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  cudaFree(lpart);
  if (e != cudaSuccess) return report_cuda_error(e, "surrogate loss/gradient");
  return MD_OK;
}

md_status md_mlp_loss_grad_device(const float* params, const float* feats, const int32_t* z,
                                  const float* target, int64_t n, float* grad, float* loss,
                                  void* stream) {
  return md::guarded([&] { return md_mlp_loss_grad_device_body(params, feats, z, target, n, grad, loss, stream); });
}

static md_status md_mlp_samples_device_body(const md_mlp_train_config* cfg, int64_t n, uint64_t seed,
                                            float* feats, int32_t* z, float* target, double* raw,
                                            void* stream) {
  md_status st = md::check_train_config(cfg);
  if (st != MD_OK) return st;
  if (n <= 0 || !feats || !z || !target) return report_error(MD_ERR_ARG, "bad sample buffers");
  md::k_mlp_samples<<<static_cast<unsigned>((n + 255) / 256), 256, 0,
                      static_cast<cudaStream_t>(stream)>>>(md::domain_io(*cfg), n, seed, feats, z,
                                                           target, raw);
  MLP_CUDA(cudaGetLastError());
  return MD_OK;
}

md_status md_mlp_samples_device(const md_mlp_train_config* cfg, int64_t n, uint64_t seed,
                                float* feats, int32_t* z, float* target, double* raw,
                                void* stream) {
  return md::guarded([&] { return md_mlp_samples_device_body(cfg, n, seed, feats, z, target, raw, stream); });
}

static md_status md_ion_rates_device_body(const md_mlp_train_config* cfg, int32_t model, const float* params,
                                          const double* emag, const int32_t* z, const double* ne,
                                          const double* te, int64_t n, double* nu, void* stream) {
  md_status st = md::check_train_config(cfg);
  if (st != MD_OK) return st;
  if (model != 1 && model != 2) return report_error(MD_ERR_ARG, "model must be 1 or 2");
  if (n < 0) return report_error(MD_ERR_ARG, "n < 0");
  if (n == 0) return MD_OK;
  if (!emag || !z || !ne || !te || !nu || (model == 2 && !params))
    return report_error(MD_ERR_ARG, "NULL pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const md::IonDev io = md::domain_io(*cfg);
  if (model == 2) {
    const long long tiles = (n + 15) / 16;
    const unsigned grid = static_cast<unsigned>(
        std::min<long long>((tiles + md::kWarps - 1) / md::kWarps, 8192));
    md::k_rates_mlp<<<grid, 32 * md::kWarps, 0, s>>>(io, params, emag, z, ne, te, n, nu);
    MLP_CUDA(cudaGetLastError());
  }
  md::k_rates_plain<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(io, emag, z, ne, te, n,
                                                                          nu, model == 1);
  MLP_CUDA(cudaGetLastError());
  return MD_OK;
}

md_status md_ion_rates_device(const md_mlp_train_config* cfg, int32_t model, const float* params,
                              const double* emag, const int32_t* z, const double* ne,
                              const double* te, int64_t n, double* nu, void* stream) {
  return md::guarded([&] { return md_ion_rates_device_body(cfg, model, params, emag, z, ne, te, n, nu, stream); });
}

static md_status md_mlp_train_body(const md_mlp_train_config* cfg, float* params_out, md_mlp_report* rep,
                                   void* stream) {
  md_status st = md::check_train_config(cfg);
  if (st != MD_OK) return st;
  if (!params_out) return report_error(MD_ERR_ARG, "params_out is NULL");
  if (cfg->n_samples < 1024 || cfg->batch < 64 || cfg->epochs < 1 || !(cfg->lr > 0.0))
    return report_error(MD_ERR_ARG, "need n_samples >= 1024, batch >= 64, epochs >= 1, lr > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MLP_CUDA(md::train_smem_attr());
  const long long n = cfg->n_samples;
  const long long nh = std::max<long long>(4096, n / 20);  // held-out set
  // one CTA per tile of the minibatch (up to two per SM): more CTAs would only
  // add zero partials for the Adam kernel to sum
  const int grid = static_cast<int>(std::max<long long>(1, std::min<long long>(
      md::train_grid(), (cfg->batch + md::kTileSamples - 1) / md::kTileSamples)));
  float *feats = nullptr, *target = nullptr, *hfeats = nullptr, *htarget = nullptr, *hy = nullptr;
  int *zs = nullptr, *hz = nullptr;
  float *p = nullptr, *m = nullptr, *v = nullptr, *part = nullptr, *lpart = nullptr,
        *lsum = nullptr;
  auto release = [&]() {
    cudaFree(feats); cudaFree(target); cudaFree(zs); cudaFree(hfeats); cudaFree(htarget);
    cudaFree(hz); cudaFree(hy); cudaFree(p); cudaFree(m); cudaFree(v); cudaFree(part);
    cudaFree(lpart); cudaFree(lsum);
  };
  bool ok = cudaMalloc(&feats, sizeof(float) * 4 * n) == cudaSuccess &&
            cudaMalloc(&target, sizeof(float) * n) == cudaSuccess &&
            cudaMalloc(&zs, sizeof(int) * n) == cudaSuccess &&
            cudaMalloc(&hfeats, sizeof(float) * 4 * nh) == cudaSuccess &&
            cudaMalloc(&htarget, sizeof(float) * nh) == cudaSuccess &&
            cudaMalloc(&hz, sizeof(int) * nh) == cudaSuccess &&
            cudaMalloc(&hy, sizeof(float) * 8 * nh) == cudaSuccess &&
            cudaMalloc(&p, sizeof(float) * md::kNParam) == cudaSuccess &&
            cudaMalloc(&m, sizeof(float) * md::kNParam) == cudaSuccess &&
            cudaMalloc(&v, sizeof(float) * md::kNParam) == cudaSuccess &&
            cudaMalloc(&part, sizeof(float) * grid * md::kNParam) == cudaSuccess &&
            cudaMalloc(&lpart, sizeof(float) * grid) == cudaSuccess &&
            cudaMalloc(&lsum, sizeof(float)) == cudaSuccess;
  if (!ok) {
    release();
    return report_error(MD_ERR_OOM, "surrogate training buffers");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  const md::IonDev io = md::domain_io(*cfg);
  md::k_mlp_samples<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(io, n, cfg->seed, feats,
                                                                          zs, target, nullptr);
  md::k_mlp_samples<<<static_cast<unsigned>((nh + 255) / 256), 256, 0, s>>>(
      io, nh, cfg->seed ^ 0x9E3779B97F4A7C15ull, hfeats, hz, htarget, nullptr);
  md::k_mlp_init<<<(md::kNParam + 255) / 256, 256, 0, s>>>(p, cfg->seed);
  cudaMemsetAsync(m, 0, sizeof(float) * md::kNParam, s);
  cudaMemsetAsync(v, 0, sizeof(float) * md::kNParam, s);
  const long long batches = (n + cfg->batch - 1) / cfg->batch;
  const long long total = batches * cfg->epochs;
  std::vector<double> losses;
  long long step = 0;
  cudaError_t e = cudaGetLastError();
  for (int ep = 0; ep < cfg->epochs && e == cudaSuccess; ++ep) {
    for (long long b = 0; b < batches && e == cudaSuccess; ++b) {
      const long long b0 = b * cfg->batch;
      const long long nb = std::min<long long>(cfg->batch, n - b0);
      ++step;
      // cosine decay of the learning rate to 1 % at the end
      const double prog = (step - 1) / static_cast<double>(total);
      const float lr = static_cast<float>(cfg->lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(3.14159265358979323846 * prog))));
      md::k_mlp_train<<<grid, 32 * md::kWarps, sizeof(md::TrainSmem), s>>>(p, feats, zs, target,
                                                                           b0, nb, part, lpart);
      md::k_mlp_adam<<<(md::kNParam + 255) / 256, 256, 0, s>>>(p, m, v, part, grid, lr, 0.9f,
                                                              0.999f, 1e-8f,
                                                              static_cast<int>(step), nullptr);
      e = cudaGetLastError();
      if (b == batches - 1 || (ep == 0 && b == 0)) {
        md::k_sum_floats<<<1, 1, 0, s>>>(lpart, grid, lsum);
        float l = 0.0f;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&l, lsum, sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        losses.push_back(l / static_cast<double>(nb));
      }
    }
  }
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) {
    md::k_mlp_forward<<<std::min<long long>((nh / 16 + md::kWarps) / md::kWarps + 1, 4096),
                        32 * md::kWarps, 0, s>>>(p, hfeats, nh, hy);
    e = cudaGetLastError();
  }
  std::vector<float> h_y(8 * nh), h_t(nh);
  std::vector<int> h_z(nh);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_y.data(), hy, sizeof(float) * 8 * nh, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_t.data(), htarget, sizeof(float) * nh, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_z.data(), hz, sizeof(int) * nh, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(params_out, p, sizeof(float) * md::kNParam, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (e != cudaSuccess) return report_cuda_error(e, "surrogate training");
  if (rep) {
    std::vector<double> d(nh);
    for (long long k = 0; k < nh; ++k)
      d[k] = 6.0 * std::fabs(static_cast<double>(h_y[8 * k + h_z[k]]) - h_t[k]);  // decades
    std::vector<double> sorted = d;
    std::sort(sorted.begin(), sorted.end());
    rep->loss_first = losses.empty() ? 0.0 : losses.front();
    rep->loss_last = losses.empty() ? 0.0 : losses.back();
    rep->holdout_median_dlog10 = sorted[nh / 2];
    rep->holdout_p99_dlog10 = sorted[static_cast<long long>(0.99 * (nh - 1))];
    rep->holdout_max_dlog10 = sorted.back();
    rep->train_ms = ms;
    rep->n_holdout = nh;
    rep->steps = step;
  }
  return MD_OK;
}

md_status md_mlp_train(const md_mlp_train_config* cfg, float* params_out, md_mlp_report* rep,
                       void* stream) {
  return md::guarded([&] { return md_mlp_train_body(cfg, params_out, rep, stream); });
}

}  // extern "C"
