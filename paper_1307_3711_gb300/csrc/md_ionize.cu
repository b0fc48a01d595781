// md_ionize.cu -- Monte-Carlo ionization pass on the GPU (Holkundkar,
// arXiv:1307.3711, Sec. II, ionization paragraph).
//
// Kernels of one cluster's pass, in launch order:
//   k_ion_field   for every ion/atom record and source segment: the Coulomb
//                 field of the live records (the TMA-staged FP32/Kahan direct
//                 sum of the step kernel) and the weight, momentum and
//                 momentum-square sums of the electrons within r_loc (from the
//                 FP32 velocity stream, landed beside the position tiles);
//   k_ion_inputs  per ion: the segments added in order, laser field at t_n,
//                 |E|, local density and temperature;
//   (k_ion_mlp_rates, md_mlp.cu: surrogate rates where the model has them)
//   k_ion_decide  per ion: total rate (static ADK + Lotz, or the surrogate's),
//                 P = 1 - exp(-nu dt_ion) and a Philox4x32-10 draw;
//   k_ion_apply   one CTA per 256 ions: the ions that fired, in index order,
//                 get charge z + 1 and free their electrons into the next free
//                 slots (a scan of the fired flags gives each its slot), so
//                 the active slots stay one dense block;
//   k_ion_fix     (a pass before every step) the field of the pass's charge
//                 changes at every ion, by segments of the changes;
//   k_ion_fix_combine  the segments added in order to each ion's field, which
//                 k_push_ions then uses to push the ions in place of the step
//                 kernel's sum.
// The decision runs after the whole field pass, so no charge changes while
// any other ion's field is being summed.  Rates are FP64, as on the host.
#include <algorithm>
#include <cmath>

#include "md_device.cuh"
#include "md_internal.h"

namespace md {

namespace {

using rate::kMeC2Ev;
using rate::kPi;

__device__ __forceinline__ bool pass_active(const IonArgs& a, long long step) {
  if (a.ion.rate_model == 0) return false;
  if (a.force) return true;
  return a.ion.ionize_every > 0 && (step % a.ion.ionize_every) == 0;
}

// --------------------------------------------------------- field + moments

// Source tiles of the ionization pass: positions/charges and, for the same
// records, the FP32 velocity stream, landed by two bulk copies on one barrier.
template <int TILE, int STAGES>
struct IonStage {
  alignas(128) float4 pos[STAGES][TILE];
  alignas(128) float4 vel[STAGES][TILE];
  alignas(8) uint64_t full[STAGES];
};

template <int TILE, int STAGES>
__device__ __forceinline__ void issue_ion_tile(IonStage<TILE, STAGES>& sm, unsigned g,
                                               const float4* pos, const float4* vel, long long ns,
                                               int t) {
  const int s = static_cast<int>(g % STAGES);
  const long long j0 = static_cast<long long>(t) * TILE;
  const long long rem = ns - j0;
  const uint32_t bytes = static_cast<uint32_t>(rem < TILE ? rem : TILE) * 16u;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&sm.full[s], 2u * bytes);
  bulk_g2s(&sm.pos[s][0], pos + j0, bytes, &sm.full[s]);
  bulk_g2s(&sm.vel[s][0], vel + j0, bytes, &sm.full[s]);
}

// Local electron moments of R ion targets: FP32 sums of w, w du and w du^2
// with du = u - u_ref, u_ref the velocity of the first electron found within
// r_loc (in source order).  The variance is unchanged by the shift, and
// centring the sums keeps the thermal spread from cancelling against a common
// drift.
template <int R>
struct LocalMoments {
  float w[R], sx[R], sy[R], sz[R], sq[R], rx[R], ry[R], rz[R];
  bool have[R];

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      w[r] = sx[r] = sy[r] = sz[r] = sq[r] = rx[r] = ry[r] = rz[r] = 0.0f;
      have[r] = false;
    }
  }
  // electron velocity record v = (ux, uy, uz, w) within r_loc of target r
  __device__ __forceinline__ void add(int r, const float4 v) {
    if (!have[r]) {
      rx[r] = v.x;
      ry[r] = v.y;
      rz[r] = v.z;
      have[r] = true;
    }
    const float ux = v.x - rx[r], uy = v.y - ry[r], uz = v.z - rz[r];
    w[r] += v.w;
    sx[r] = fmaf(v.w, ux, sx[r]);
    sy[r] = fmaf(v.w, uy, sy[r]);
    sz[r] = fmaf(v.w, uz, sz[r]);
    sq[r] = fmaf(v.w, fmaf(ux, ux, fmaf(uy, uy, uz * uz)), sq[r]);
  }
};

// Charge class of a landed tile (same answer in every warp): one charge for
// all its sources or not, and whether any source is an electron (q < 0).
__device__ __forceinline__ void tile_class(uint32_t tile, int cnt, float& q, bool& uniform,
                                           bool& has_electron) {
  q = lds_f32(tile + 12u);
  bool ok = true, neg = false;
  for (int k = static_cast<int>(threadIdx.x & 31u); k < cnt; k += 32) {
    const float w = lds_f32(tile + 16u * k + 12u);
    ok = ok && (w == q);
    neg = neg || (w < 0.0f);
  }
  uniform = __all_sync(0xffffffffu, ok);
  has_electron = __any_sync(0xffffffffu, neg);
}

// Pairs of one tile with the local moments.  UNIFORM: every source is an
// electron of one charge, the charge is applied once per tile (fold_q);
// otherwise each pair takes its own charge and only electrons count.
// rloc2e = r_loc^2 + eps^2 is compared with r^2 + eps^2.  Sources go in
// groups of 4 with one (rarely taken) branch per group on the nearest of the
// 4; inside it the electrons within r_loc are added in source order.
template <int R, bool UNIFORM, bool MI = false>
__device__ __forceinline__ void ion_pairs_moments(uint32_t ptile, const float4* vtile, int cnt,
                                                  const float (&xi)[R], const float (&yi)[R],
                                                  const float (&zi)[R], float eps2, float rloc2e,
                                                  Acc<R, false>& acc, LocalMoments<R>& m,
                                                  float L = 0.0f, float invL = 0.0f) {
  constexpr int G = 4;
  int j = 0;
  for (; j + G <= cnt; j += G) {
    float4 p[G];
#pragma unroll
    for (int g = 0; g < G; ++g) p[g] = lds_f4(ptile + 16u * (j + g));
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float near2[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        float dx = p[g].x - xi[r], dy = p[g].y - yi[r], dz = p[g].z - zi[r];
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
        const float s3 = UNIFORM ? ri2 * ri : p[g].w * ri2 * ri;
        acc.ax[r] = fmaf(dx, s3, acc.ax[r]);
        acc.ay[r] = fmaf(dy, s3, acc.ay[r]);
        acc.az[r] = fmaf(dz, s3, acc.az[r]);
        near2[g] = (UNIFORM || p[g].w < 0.0f) ? r2 : rloc2e;
      }
      const float mn = fminf(fminf(near2[0], near2[1]), fminf(near2[2], near2[3]));
      if (mn < rloc2e) {
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (near2[g] < rloc2e) m.add(r, vtile[j + g]);
      }
    }
  }
  for (; j < cnt; ++j) {
    const float4 p = lds_f4(ptile + 16u * j);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float dx = p.x - xi[r], dy = p.y - yi[r], dz = p.z - zi[r];
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
      const float s3 = UNIFORM ? ri2 * ri : p.w * ri2 * ri;
      acc.ax[r] = fmaf(dx, s3, acc.ax[r]);
      acc.ay[r] = fmaf(dy, s3, acc.ay[r]);
      acc.az[r] = fmaf(dz, s3, acc.az[r]);
      if ((UNIFORM || p.w < 0.0f) && r2 < rloc2e) m.add(r, vtile[j]);
    }
  }
}

// One landed tile of the field pass (the dispatch of k_ion_field by the
// tile's charge class), for the minimum-image twin, which picks MI per tile.
template <int R, bool MI>
__device__ __forceinline__ void ion_tile(uint32_t ptile, const float4* vtile, int cnt,
                                         const float (&xi)[R], const float (&yi)[R],
                                         const float (&zi)[R], float eps2, float rloc2e,
                                         Acc<R, false>& acc, LocalMoments<R>& mom, float L,
                                         float invL) {
  float qt;
  bool uniform, has_e;
  tile_class(ptile, cnt, qt, uniform, has_e);
  if (uniform) {
    if (qt < 0.0f) {
      ion_pairs_moments<R, true, MI>(ptile, vtile, cnt, xi, yi, zi, eps2, rloc2e, acc, mom, L,
                                     invL);
      fold_q<R, false>(acc, qt);
    } else if (qt > 0.0f) {
#pragma unroll 4
      for (int j = 0; j < cnt; ++j)
        pair_u<R, false, MI>(lds_f4(ptile + 16u * j), xi, yi, zi, eps2, acc, L, invL);
      fold_q<R, false>(acc, qt);
    }
  } else if (has_e) {
    ion_pairs_moments<R, false, MI>(ptile, vtile, cnt, xi, yi, zi, eps2, rloc2e, acc, mom, L,
                                    invL);
    fold<R, false>(acc);
  } else {
#pragma unroll 4
    for (int j = 0; j < cnt; ++j)
      pair<R, false, MI>(lds_f4(ptile + 16u * j), xi, yi, zi, eps2, acc, L, invL);
    fold<R, false>(acc);
  }
}

// Field (FP32/Kahan) and local electron moments at R ion targets per thread,
// from source segment blockIdx.y of the cluster's live records.  The live
// records are the ions and electrons below the next free electron slot (the
// slots are filled densely), split into gridDim.y equal segments.  Tiles of
// one charge take the charge out of the pair loop; ion-only tiles skip the
// moment test; uncharged tiles and dead record groups are skipped.
template <int THREADS, int R, int TILE, int STAGES, bool MI = false>
__global__ void __launch_bounds__(THREADS) k_ion_field(const IonArgs a) {
  __shared__ IonStage<TILE, STAGES> sm;
  __shared__ int s_abort;
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  // live records [0, n_live): no active electron sits at or above the next free slot
  long long n_live = __ldcg(a.next_slot);
  n_live = n_live > a.ion.slot_base ? n_live : a.ion.slot_base;
  n_live = n_live < a.c.n_pad ? (n_live > 0 ? n_live : 0) : a.c.n_pad;
  const long long per_seg = (n_live + gridDim.y - 1) / gridDim.y;
  const long long seg_len = (per_seg + TILE - 1) / TILE * TILE;
  const long long j0 = static_cast<long long>(blockIdx.y) * seg_len;
  const long long ns = (j0 >= n_live) ? 0 : ((n_live - j0 < seg_len) ? n_live - j0 : seg_len);
  const float4* src = cur + a.c.off + j0;
  const float4* vsrc = a.vel + a.c.off + j0;
  const long long t0 = static_cast<long long>(blockIdx.x) * (THREADS * R);
  const float eps2 = a.c.eps2;
  const float rloc2e = static_cast<float>(a.ion.r_loc * a.ion.r_loc) + eps2;
  float xi[R], yi[R], zi[R];
  Acc<R, false> acc;
  acc.zero();
  LocalMoments<R> mom;
  mom.zero();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = t0 + threadIdx.x + r * THREADS;
    const float4 p = (t < a.ion.n_ions) ? cur[a.c.off + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
  }
  // minimum-image twin: image distances while the boundary is periodic at t_n
  bool mi_on = false;
  float L = 0.0f, invL = 0.0f;
  [[maybe_unused]] float* s_tb = nullptr;
  if constexpr (MI) {
    __shared__ float tb[6];
    const double t_n = a.c.t0 + static_cast<double>(step) * a.c.dt;
    mi_on = a.min_image && (a.c.boundary == 1 || (a.c.boundary == 2 && t_n < a.c.t_switch));
    L = static_cast<float>(a.c.box);
    invL = 1.0f / L;
    s_tb = tb;
    if (mi_on) target_bounds<THREADS, R>(xi, yi, zi, tb);
  }
  const int ntiles = static_cast<int>((ns + TILE - 1) / TILE);
  // only tiles holding a live group are copied and summed, in the same order
  // for the issuing thread and the consumers
  const long long gb = a.c.off + j0;
  int t = next_live_tile(a.src_live, gb, ns, 0, ntiles, TILE);
  int ti = t;
  unsigned issued = 0;
  if (threadIdx.x == 0) {
    for (; issued < static_cast<unsigned>(STAGES) && ti < ntiles; ++issued) {
      issue_ion_tile<TILE, STAGES>(sm, issued, src, vsrc, ns, ti);
      ti = next_live_tile(a.src_live, gb, ns, ti + 1, ntiles, TILE);
    }
  }
  for (unsigned k = 0; t < ntiles; ++k) {
    const int s = static_cast<int>(k % STAGES);
    if (!mbar_wait(&sm.full[s], (k / STAGES) & 1u)) {
      atomicOr(a.err, kErrTimeout);
      s_abort = 1;
    }
    const long long jb = static_cast<long long>(t) * TILE;
    const long long rem = ns - jb;
    const int cnt = static_cast<int>(rem < TILE ? rem : TILE);
    if (!*reinterpret_cast<volatile int*>(&s_abort)) {
      const uint32_t ptile = smem_u32(&sm.pos[s][0]);
      if constexpr (MI) {
        // minimum-image distances only for tiles with pairs half a box apart
        if (mi_on && tile_needs_image(ptile, cnt, s_tb, L))
          ion_tile<R, true>(ptile, &sm.vel[s][0], cnt, xi, yi, zi, eps2, rloc2e, acc, mom, L,
                            invL);
        else
          ion_tile<R, false>(ptile, &sm.vel[s][0], cnt, xi, yi, zi, eps2, rloc2e, acc, mom, L,
                             invL);
      } else {
        float qt;
        bool uniform, has_e;
        tile_class(ptile, cnt, qt, uniform, has_e);
        if (uniform) {
          if (qt < 0.0f) {
            ion_pairs_moments<R, true>(ptile, &sm.vel[s][0], cnt, xi, yi, zi, eps2, rloc2e, acc,
                                       mom);
            fold_q<R, false>(acc, qt);
          } else if (qt > 0.0f) {
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) pair_u<R, false>(lds_f4(ptile + 16u * j), xi, yi, zi, eps2, acc);
            fold_q<R, false>(acc, qt);
          }
        } else if (has_e) {
          ion_pairs_moments<R, false>(ptile, &sm.vel[s][0], cnt, xi, yi, zi, eps2, rloc2e, acc,
                                      mom);
          fold<R, false>(acc);
        } else {
#pragma unroll 4
          for (int j = 0; j < cnt; ++j) pair<R, false>(lds_f4(ptile + 16u * j), xi, yi, zi, eps2, acc);
          fold<R, false>(acc);
        }
      }
    }
    __syncthreads();
    if (*reinterpret_cast<volatile int*>(&s_abort)) {
      if (threadIdx.x == 0) {
        for (unsigned q = k + 1; q < issued; ++q)
          mbar_wait(&sm.full[q % STAGES], (q / STAGES) & 1u);
      }
      return;
    }
    if (threadIdx.x == 0 && ti < ntiles) {
      issue_ion_tile<TILE, STAGES>(sm, issued, src, vsrc, ns, ti);
      ++issued;
      ti = next_live_tile(a.src_live, gb, ns, ti + 1, ntiles, TILE);
    }
    t = next_live_tile(a.src_live, gb, ns, t + 1, ntiles, TILE);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long tt = t0 + threadIdx.x + r * THREADS;
    if (tt >= a.ion.n_ions) continue;
    if (!MD_IN_RANGE(a.err, blockIdx.y, 0, kIonMaxSeg)) continue;
    double* o = a.scratch + kIonScratch * (static_cast<long long>(blockIdx.y) * a.ion.n_ions + tt);
    o[0] = -(static_cast<double>(acc.sx[r]) - acc.cx[r]);
    o[1] = -(static_cast<double>(acc.sy[r]) - acc.cy[r]);
    o[2] = -(static_cast<double>(acc.sz[r]) - acc.cz[r]);
    o[3] = mom.w[r];
    o[4] = mom.sx[r];
    o[5] = mom.sy[r];
    o[6] = mom.sz[r];
    o[7] = mom.sq[r];
    o[8] = mom.rx[r];
    o[9] = mom.ry[r];
    o[10] = mom.rz[r];
  }
}

// ------------------------------------------- field and moments, separately --
//
// Clusters without minimum-image forces take the field and the local moments
// of the pass in two parts: k_ion_field_sum sums the field of the live records
// at the ions (the step kernel's TMA source loop, no moment test in the pair
// loop), and the moments come from a cell list of the electrons near the ions,
// so each ion tests only the electrons of its own and the 26 neighbouring
// cells.  The moments are summed about the ion's own velocity: each
// electron's terms are rounded to FP32, then to 64-bit fixed point (units of
// 2^-40), and integer sums do not depend on the order in which the cells
// list their electrons, so the result is deterministic although the listing
// uses atomic counters.  The near test is the field pass's: the FP32
// r^2 + eps^2 of the j-stream positions against r_loc^2 + eps^2.

// Field of the live records at the ions: CTA (x, y) sums segment y of the
// live records for R x THREADS ions and writes its field to the scratch
// slots of segment y (slots 0-2; slot 3, the weight of the local electrons,
// is 0 here and filled for segment 0 by k_ion_moments).
template <int THREADS, int R, int TILE, int STAGES, bool PACK>
__global__ void __launch_bounds__(THREADS) k_ion_field_sum(const IonArgs a) {
  __shared__ Stage<TILE, STAGES> sm;
  __shared__ DupTile<PACK ? TILE : 1> dup;
  __shared__ KahanSmem<PACK ? R / 2 : 1, PACK ? THREADS : 1, false> ks;
  __shared__ int s_abort;
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  long long n_live = __ldcg(a.next_slot);
  n_live = n_live > a.ion.slot_base ? n_live : a.ion.slot_base;
  n_live = n_live < a.c.n_pad ? (n_live > 0 ? n_live : 0) : a.c.n_pad;
  const long long per_seg = (n_live + gridDim.y - 1) / gridDim.y;
  const long long seg_len = (per_seg + TILE - 1) / TILE * TILE;
  const long long j0 = static_cast<long long>(blockIdx.y) * seg_len;
  const long long ns = (j0 >= n_live) ? 0 : ((n_live - j0 < seg_len) ? n_live - j0 : seg_len);
  const long long t0 = static_cast<long long>(blockIdx.x) * (THREADS * R);
  float xi[R], yi[R], zi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = t0 + threadIdx.x + r * THREADS;
    const float4 p = (t < a.ion.n_ions) ? cur[a.c.off + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
  }
  Acc<R, false> acc;
  acc.zero();
  unsigned it = 0;
  if constexpr (PACK) {
    // (an empty segment still clears the Kahan sums and returns at once)
    if (!sum_sources_packed<THREADS, R, TILE, STAGES, false>(
            sm, dup, ks, it, cur + a.c.off + j0, ns, xi, yi, zi, a.c.eps2, a.err, &s_abort,
            a.src_live, a.c.off + j0))
      return;
  } else if (ns > 0) {
    if (!sum_sources<THREADS, R, TILE, STAGES, false>(sm, it, cur + a.c.off + j0, ns, xi, yi, zi,
                                                      a.c.eps2, acc, a.err, &s_abort, a.src_live,
                                                      a.c.off + j0))
      return;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long tt = t0 + threadIdx.x + r * THREADS;
    if (tt >= a.ion.n_ions) continue;
    if (!MD_IN_RANGE(a.err, blockIdx.y, 0, kIonMaxSeg)) continue;
    double* o = a.scratch + kIonScratch * (static_cast<long long>(blockIdx.y) * a.ion.n_ions + tt);
    if constexpr (PACK) {
      o[0] = -(static_cast<double>(kahan_part(ks, 0, r)) - kahan_part(ks, 3, r));
      o[1] = -(static_cast<double>(kahan_part(ks, 1, r)) - kahan_part(ks, 4, r));
      o[2] = -(static_cast<double>(kahan_part(ks, 2, r)) - kahan_part(ks, 5, r));
    } else {
      o[0] = -(static_cast<double>(acc.sx[r]) - acc.cx[r]);
      o[1] = -(static_cast<double>(acc.sy[r]) - acc.cy[r]);
      o[2] = -(static_cast<double>(acc.sz[r]) - acc.cz[r]);
    }
    o[3] = 0.0;
  }
}

// Spatial hash of the cell list: cells of side h = 1.01 r_loc, so an electron
// within r_loc of an ion lies in the ion's cell or one of the 26 around it;
// the integer cell coordinates are hashed into kCellBuckets buckets (distant
// cells may share a bucket; the near test rejects their electrons).
__device__ __forceinline__ bool cell_coords(float x, float y, float z, float inv_h, int* cc) {
  const float p[3] = {x * inv_h, y * inv_h, z * inv_h};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float f = floorf(p[c]);
    if (!(f > -1.0e9f && f < 1.0e9f)) return false;  // far away or not finite
    cc[c] = static_cast<int>(f);
  }
  return true;
}

// The three coordinates (mod 2^21) packed into one 63-bit key, hashed by
// Knuth's multiplicative method: the top bits of the key times 2^64 / phi.
// (An XOR of the coordinates times three odd constants, the first version,
// put the mirror cells (0, y, z) and (0, -y, -z) of a cluster centred on the
// origin into one bucket whenever y and z have the same power of 2.)
__device__ __forceinline__ int cell_bucket(int x, int y, int z) {
  constexpr unsigned long long kMask = (1ull << 21) - 1;
  const unsigned long long key = (static_cast<unsigned long long>(x) & kMask) |
                                 ((static_cast<unsigned long long>(y) & kMask) << 21) |
                                 ((static_cast<unsigned long long>(z) & kMask) << 42);
  constexpr int kBits = 18;
  static_assert(kCellBuckets == 1 << kBits, "bucket count");
  return static_cast<int>((key * 0x9E3779B97F4A7C15ull) >> (64 - kBits));
}

__device__ __forceinline__ int bucket_of(float x, float y, float z, float inv_h) {
  int cc[3];
  if (!cell_coords(x, y, z, inv_h, cc)) return -1;
  return cell_bucket(cc[0], cc[1], cc[2]);
}

__device__ __forceinline__ float cell_inv_h(const IonArgs& a) {
  return 1.0f / (1.01f * static_cast<float>(a.ion.r_loc));
}

// FILL = false: count the electrons (negative charge) of the live records per
// cell; FILL = true: list each at its cell's start + an atomic fill counter.
template <bool FILL>
__global__ void __launch_bounds__(256) k_cell_list(const IonArgs a) {
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  long long n_live = __ldcg(a.next_slot);
  n_live = n_live > a.ion.slot_base ? n_live : a.ion.slot_base;
  n_live = n_live < a.c.n_pad ? (n_live > 0 ? n_live : 0) : a.c.n_pad;
  const CellBuf cb = a.cells;
  const float inv_h = cell_inv_h(a);
  for (long long j = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; j < n_live;
       j += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float4 p = cur[a.c.off + j];
    if (!(p.w < 0.0f)) continue;
    const int cell = bucket_of(p.x, p.y, p.z, inv_h);
    if (cell < 0) continue;
    if (!FILL) {
      atomicAdd(cb.count + cell, 1);
    } else {
      const long long k = cb.start[cell] + atomicAdd(cb.fill + cell, 1);
      if (!MD_IN_RANGE(a.err, k, 0, cb.capacity)) continue;
      cb.rec[2 * k] = p;
      cb.rec[2 * k + 1] = a.vel[a.c.off + j];
    }
  }
}

// FILL = false: count the ions per cell; FILL = true: list them in cell order.
template <bool FILL>
__global__ void __launch_bounds__(256) k_ion_cell_list(const IonArgs a) {
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  const CellBuf cb = a.cells;
  const float inv_h = cell_inv_h(a);
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
       t < a.ion.n_ions; t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float4 p = cur[a.c.off + t];
    int cell = bucket_of(p.x, p.y, p.z, inv_h);
    if (cell < 0) cell = 0;  // a position too far away to have a cell: its moments stay 0
    if (!FILL) {
      atomicAdd(cb.ion_count + cell, 1);
    } else {
      const long long k = cb.ion_start[cell] + atomicAdd(cb.ion_fill + cell, 1);
      if (!MD_IN_RANGE(a.err, k, 0, a.ion.n_ions)) continue;
      cb.ion_list[k] = static_cast<int>(t);
    }
  }
}

// Exclusive scan of the kCellBuckets bucket counts into starts, in three
// launches: each of kScanBlocks CTAs scans its 1024 buckets and records their
// total; one CTA scans the totals; each CTA adds its offset.
constexpr int kScanBlocks = kCellBuckets / 1024;

__device__ __forceinline__ int block_excl_scan_1024(int v, int* s_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = s_warp[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    s_warp[lane] = w;  // inclusive scan of the warp totals
  }
  __syncthreads();
  const int before = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
  if (total) *total = s_warp[31];
  return before;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(const IonArgs a, const int* count,
                                                      int* start, int* totals) {
  __shared__ int s_warp[32];
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const int k = blockIdx.x * 1024 + threadIdx.x;
  int tot = 0;
  start[k] = block_excl_scan_1024(count[k], s_warp, &tot);
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_totals(const IonArgs a, int* totals, int* start) {
  __shared__ int s_warp[32];
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const int v = threadIdx.x < kScanBlocks ? totals[threadIdx.x] : 0;
  int tot = 0;
  const int before = block_excl_scan_1024(v, s_warp, &tot);
  __syncthreads();
  if (threadIdx.x < kScanBlocks) totals[threadIdx.x] = before;
  if (threadIdx.x == 0) start[kCellBuckets] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_add(const IonArgs a, const int* totals,
                                                   int* start) {
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  start[blockIdx.x * 1024 + threadIdx.x] += totals[blockIdx.x];
}

cudaError_t launch_cell_scan(const IonArgs& a, const int* count, int* start, cudaStream_t s) {
  k_scan_blocks<<<kScanBlocks, 1024, 0, s>>>(a, count, start, a.cells.scan_tmp);
  k_scan_totals<<<1, 1024, 0, s>>>(a, a.cells.scan_tmp, start);
  k_scan_add<<<kScanBlocks, 1024, 0, s>>>(a, a.cells.scan_tmp, start);
  return cudaGetLastError();
}

// Local moments of every ion from the electrons of its 27 cells (R14): weight
// W, and about u_ref = the ion's own velocity the sums S = sum w du and
// Q = sum w |du|^2, in fixed point; written as segment 0 of the scratch.
// Each electron's terms are rounded to FP32 and then exactly to 2^-40 units
// and added to 64-bit integer sums, so a total does not depend on which lane
// took which electron, nor on the order of the listing.
//
// The ions are taken in bucket order, kMomIons per CTA.  The ions of one
// bucket mostly share one cell and so one set of 27 neighbour cells: for each
// run of ions with the same bucket, the positions of the electrons listed in
// those cells' buckets (a few thousand) are staged once in shared memory, and
// each warp tests them against one ion at a time, 32 electrons per step.  An
// ion of the run in another cell (two cells hashed to one bucket, or a
// position without a cell) and a run whose electrons do not fit the stage
// walk their own 27 buckets from global memory instead.
constexpr int kMomThreads = 256;
constexpr int kMomWarps = kMomThreads / 32;
constexpr int kMomIons = 64;     // ions per CTA
constexpr int kMomCap = 3072;    // staged electrons per run

// v rounded to the nearest integer, ties to even, as a 64-bit integer, on
// the integer pipe (for |v| < 2^62).  From the binary32 layout: v = m 2^s
// with the 24-bit significand m and s = exponent - 150; for s >= 0 the value
// is m shifted left, else m / 2^-s rounded by its remainder (every |v| < 1/2
// rounds to 0, so the shift stops at 25).  GB300 runs the F2I.S64 conversion
// on its narrow FP64 pipe, which held it 85 % busy in this kernel.
__device__ __forceinline__ long long rint_ll(float v) {
  const unsigned b = __float_as_uint(v);
  const int e = static_cast<int>((b >> 23) & 0xffu);
  const unsigned long long m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
  const int s = e - 150;
  unsigned long long r;
  if (s >= 0) {
    r = m << (s < 62 ? s : 62);
  } else {
    const int k = -s < 25 ? -s : 25;
    const unsigned long long q = m >> k, rem = m & ((1ull << k) - 1), half = 1ull << (k - 1);
    r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  }
  const long long x = static_cast<long long>(r);
  return (b >> 31) ? -x : x;
}

struct MomSums {
  long long W = 0, S0 = 0, S1 = 0, S2 = 0, Q = 0;

  // one electron of velocity record v (w in .w) against an ion of velocity ui
  __device__ __forceinline__ void add(const float4 v, const float4 ui) {
    constexpr float kScaleF = 1099511627776.0f;  // 2^40
    const float ux = v.x - ui.x, uy = v.y - ui.y, uz = v.z - ui.z;
    const float ws = v.w * kScaleF;
    W += rint_ll(ws);
    S0 += rint_ll(ws * ux);
    S1 += rint_ll(ws * uy);
    S2 += rint_ll(ws * uz);
    Q += rint_ll(ws * fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
  }

  __device__ __forceinline__ void warp_sum() {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      W += __shfl_xor_sync(0xffffffffu, W, d);
      S0 += __shfl_xor_sync(0xffffffffu, S0, d);
      S1 += __shfl_xor_sync(0xffffffffu, S1, d);
      S2 += __shfl_xor_sync(0xffffffffu, S2, d);
      Q += __shfl_xor_sync(0xffffffffu, Q, d);
    }
  }
};

__device__ __forceinline__ bool near_loc(const float4 p, const float4 pi, float eps2,
                                         float rloc2e) {
  const float ddx = p.x - pi.x, ddy = p.y - pi.y, ddz = p.z - pi.z;
  float r2 = fmaf(ddx, ddx, eps2);
  r2 = fmaf(ddy, ddy, r2);
  r2 = fmaf(ddz, ddz, r2);
  return r2 < rloc2e;
}

// Lane l < 27 of a warp: the bucket of neighbour cell l of cc (offsets
// l % 3 - 1, l / 3 % 3 - 1, l / 9 - 1), or -1 for a repeat of a lower lane's
// bucket (cells may share one) and for lanes 27..31.
__device__ __forceinline__ int neighbour_bucket(const int (&cc)[3], int lane) {
  int bk = -1;
  if (lane < 27)
    bk = cell_bucket(cc[0] + lane % 3 - 1, cc[1] + (lane / 3) % 3 - 1, cc[2] + lane / 9 - 1);
  bool first = lane < 27;
  for (int m = 0; m < 27; ++m) {
    const int bm = __shfl_sync(0xffffffffu, bk, m);
    if (m < lane && bm == bk) first = false;
  }
  return first ? bk : -1;
}

// One warp: the sums of one ion over its 27 cells' buckets, read from global
// memory (lane-strided over each bucket's electrons).
__device__ __forceinline__ void moments_global(const CellBuf& cb, const float4 pi,
                                               const float4 ui, const int (&cc)[3], float eps2,
                                               float rloc2e, int lane, MomSums& m, int* err) {
  const int bk = neighbour_bucket(cc, lane);
  unsigned todo = __ballot_sync(0xffffffffu, bk >= 0);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const int cell = __shfl_sync(0xffffffffu, bk, src);
    const int k1 = cb.start[cell + 1];
    for (int k = cb.start[cell] + lane; k < k1; k += 32)
      if (MD_IN_RANGE(err, k, 0, cb.capacity) && near_loc(cb.rec[2 * k], pi, eps2, rloc2e))
        m.add(cb.rec[2 * k + 1], ui);
  }
}

__global__ void __launch_bounds__(kMomThreads) k_ion_moments(const IonArgs a) {
  __shared__ float4 s_pos[kMomCap];
  __shared__ int s_idx[kMomCap];
  // per warp: the electrons found within r_loc and not yet added, so that
  // the terms are added 32 at a time with every lane busy
  __shared__ int s_near[kMomWarps][64];
  __shared__ int s_bucket[kMomIons];
  __shared__ int s_bk[32], s_beg[32], s_cnt[32];
  __shared__ int s_total;
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const CellBuf cb = a.cells;
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  const float eps2 = a.c.eps2;
  const float rloc2e = static_cast<float>(a.ion.r_loc * a.ion.r_loc) + eps2;
  const float inv_h = cell_inv_h(a);
  const long long c0 = static_cast<long long>(blockIdx.x) * kMomIons;
  const int nloc = static_cast<int>(a.ion.n_ions - c0 < kMomIons ? a.ion.n_ions - c0 : kMomIons);
  // each ion's bucket, as the ion listing computed it (no cell: bucket 0)
  if (tid < nloc) {
    const long long t = cb.ion_list[c0 + tid];
    int b = 0;
    if (MD_IN_RANGE(a.err, t, 0, a.ion.n_ions)) {
      const float4 p = cur[a.c.off + t];
      b = bucket_of(p.x, p.y, p.z, inv_h);
      b = b < 0 ? 0 : b;
    }
    s_bucket[tid] = b;
  }
  __syncthreads();
  for (int r0 = 0; r0 < nloc;) {
    int r1 = r0 + 1;
    while (r1 < nloc && s_bucket[r1] == s_bucket[r0]) ++r1;
    // the run's first ion sets the staged cell
    const long long t0 = cb.ion_list[c0 + r0];
    int cc0[3] = {0, 0, 0};
    bool staged = MD_IN_RANGE(a.err, t0, 0, a.ion.n_ions);
    if (staged) {
      const float4 p0 = cur[a.c.off + t0];
      staged = cell_coords(p0.x, p0.y, p0.z, inv_h, cc0);
    }
    if (staged && warp == 0) {
      const int bk = neighbour_bucket(cc0, lane);
      const int cnt = bk >= 0 ? cb.start[bk + 1] - cb.start[bk] : 0;
      int inc = cnt;  // inclusive scan of the counts over the lanes
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
      }
      s_bk[lane] = bk;
      s_cnt[lane] = cnt;
      s_beg[lane] = inc - cnt;
      if (lane == 31) s_total = inc;
    }
    __syncthreads();
    staged = staged && s_total <= kMomCap;
    if (staged) {
      for (int l = 0; l < 27; ++l) {
        const int cnt = s_cnt[l];
        if (cnt == 0) continue;
        const int k0 = cb.start[s_bk[l]], beg = s_beg[l];
        for (int k = tid; k < cnt; k += kMomThreads) {
          const bool ok = MD_IN_RANGE(a.err, k0 + k, 0, cb.capacity);
          // (an index out of range stages a position no ion is near)
          s_pos[beg + k] = ok ? cb.rec[2 * (k0 + k)] : make_float4(3e38f, 3e38f, 3e38f, 0.f);
          s_idx[beg + k] = ok ? k0 + k : 0;
        }
      }
    }
    __syncthreads();
    const int total = staged ? s_total : 0;
    for (int q = r0 + warp; q < r1; q += kMomWarps) {
      const long long t = cb.ion_list[c0 + q];
      if (!MD_IN_RANGE(a.err, t, 0, a.ion.n_ions)) continue;  // warp-uniform
      const float4 pi = cur[a.c.off + t];
      const float4 ui = a.vel[a.c.off + t];
      MomSums m;
      int cc[3];
      if (cell_coords(pi.x, pi.y, pi.z, inv_h, cc)) {
        if (staged && cc[0] == cc0[0] && cc[1] == cc0[1] && cc[2] == cc0[2]) {
          int* q = s_near[warp];
          int qn = 0;  // queued electrons (warp-uniform)
          for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            const bool nr = k < total && near_loc(s_pos[k], pi, eps2, rloc2e);
            const unsigned mask = __ballot_sync(0xffffffffu, nr);
            if (nr) q[qn + __popc(mask & ((1u << lane) - 1u))] = s_idx[k];
            qn += __popc(mask);
            if (qn >= 32) {
              __syncwarp();
              m.add(cb.rec[2 * q[lane] + 1], ui);
              const int rest = qn - 32 > lane ? q[32 + lane] : 0;
              __syncwarp();
              if (lane < qn - 32) q[lane] = rest;
              __syncwarp();
              qn -= 32;
            }
          }
          __syncwarp();
          if (lane < qn) m.add(cb.rec[2 * q[lane] + 1], ui);
          __syncwarp();
        } else {
          moments_global(cb, pi, ui, cc, eps2, rloc2e, lane, m, a.err);
        }
        m.warp_sum();
      }
      if (lane == 0) {
        constexpr double kScale = 1099511627776.0;  // 2^40
        double* o = a.scratch + kIonScratch * t;  // segment 0
        o[3] = static_cast<double>(m.W) / kScale;
        o[4] = static_cast<double>(m.S0) / kScale;
        o[5] = static_cast<double>(m.S1) / kScale;
        o[6] = static_cast<double>(m.S2) / kScale;
        o[7] = static_cast<double>(m.Q) / kScale;
        o[8] = ui.x;
        o[9] = ui.y;
        o[10] = ui.z;
      }
    }
    __syncthreads();  // the stage is rewritten by the next run
    r0 = r1;
  }
}

// ------------------------------------------------------------- decision --

__device__ __forceinline__ double laser_ax(const ClusterDev& c, double t, double* ay) {
  const double amp = c.a0 * envelope(t, c.env, c.tau);
  double sn, cs;
  sincos(t, &sn, &cs);
  *ay = c.pol ? -amp * cs : 0.0;
  return amp * sn;
}

// Per ion: total field with the laser at t_n, local density and temperature.
__global__ void __launch_bounds__(256) k_ion_inputs(const IonArgs a) {
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= a.ion.n_ions) return;
  if (t == 0) *a.pass_slot = *a.next_slot;  // the apply kernel's base for this pass
  // combine the source segments in order: fields add; the moments of each
  // segment are shifted to the reference of the first segment with electrons
  // (sums about r_s -> sums about r: S += W d, Q += 2 d.S + W |d|^2, d = r_s - r)
  double fx = 0.0, fy = 0.0, fz = 0.0, W = 0.0, S[3] = {0.0, 0.0, 0.0}, Q = 0.0, ref[3];
  bool have = false;
  for (int sg = 0; sg < a.nseg; ++sg) {
    const double* sc = a.scratch + kIonScratch * (static_cast<long long>(sg) * a.ion.n_ions + t);
    fx += sc[0];
    fy += sc[1];
    fz += sc[2];
    if (!(sc[3] > 0.0)) continue;
    if (!have) {
      ref[0] = sc[8]; ref[1] = sc[9]; ref[2] = sc[10];
      have = true;
    }
    const double d0 = sc[8] - ref[0], d1 = sc[9] - ref[1], d2 = sc[10] - ref[2];
    Q += sc[7] + 2.0 * (d0 * sc[4] + d1 * sc[5] + d2 * sc[6]) + sc[3] * (d0 * d0 + d1 * d1 + d2 * d2);
    S[0] += sc[4] + sc[3] * d0;
    S[1] += sc[5] + sc[3] * d1;
    S[2] += sc[6] + sc[3] * d2;
    W += sc[3];
  }
  if (a.e_ion) {
    a.e_ion[3 * t + 0] = fx;
    a.e_ion[3 * t + 1] = fy;
    a.e_ion[3 * t + 2] = fz;
  }
  const double tn = a.c.t0 + static_cast<double>(step) * a.c.dt;
  double lay;
  const double lax = laser_ax(a.c, tn, &lay);
  const double ex = fx + lax, ey = fy + lay, ez = fz;
  double ne = 0.0, te = 0.0;
  if (W > 0.0) {
    const double lk = a.ion.r_loc / a.ion.k_si;  // r_loc in metres
    const double vol_cm3 = (4.0 / 3.0) * kPi * lk * lk * lk * 1e6;
    const double mx = S[0] / W, my = S[1] / W, mz = S[2] / W;
    const double var = Q / W - (mx * mx + my * my + mz * mz);
    ne = W / vol_cm3;
    te = var > 0.0 ? kMeC2Ev * var / 3.0 : 0.0;
  }
  double* o = a.out + 4 * t;
  o[0] = sqrt(ex * ex + ey * ey + ez * ez);
  o[1] = ne;
  o[2] = te;
  o[3] = 0.0;
  a.nu[t] = -1.0;
}

// Per ion: rate (surrogate if it set one, else static ADK + Lotz), P and the
// Philox draw; sets fired[t] and the number of fired ions of the block.  No
// state changes here.
__global__ void __launch_bounds__(256) k_ion_decide(const IonArgs a) {
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  int fired = 0;
  if (t < a.ion.n_ions) {
    const long long i = a.c.off + t;
    double* o = a.out + 4 * t;
    const int z = a.zq[i];
    if (a.kind[i] == 0 && z >= 0 && z < a.ion.zmax) {
      const double emag = o[0], ne = o[1], te = o[2];
      const double nu_s = a.nu[t];
      const double nu = nu_s >= 0.0 ? nu_s : rate::rate_plain(a.ion, emag, z, ne, te);
      const double dt_ion = (a.ion.ionize_every > 0 ? a.ion.ionize_every : 1) * a.c.dt;
      const double P = -expm1(-nu * dt_ion);
      o[3] = P;
      const uint4 wv = philox4x32_10(
          make_uint4(static_cast<uint32_t>(t), static_cast<uint32_t>(step),
                     static_cast<uint32_t>(static_cast<unsigned long long>(step) >> 32), 0u),
          make_uint2(static_cast<uint32_t>(a.ion.seed), static_cast<uint32_t>(a.ion.seed >> 32)));
      const double alpha = (static_cast<double>(wv.x) + 1.0) * (1.0 / 4294967296.0);
      fired = alpha < P ? 1 : 0;
    }
    a.fired[t] = static_cast<unsigned char>(fired);
  }
  const int cnt = __syncthreads_count(fired);
  if (threadIdx.x == 0) a.blk_fired[blockIdx.x] = cnt;
}

// Ionization of ion t (cluster-relative) freeing its electron into record e
// (cluster-relative): charge update, the electron uniform in the ball of
// radius r_create around the ion (Philox words 1-3 of the decision's draw)
// with the ion's u and weight, liveness flags.
__device__ void apply_one(const IonArgs& a, long long step, long long t, long long e_rel) {
  const long long i = a.c.off + t;
  const int z = a.zq[i];
  const int z1 = z + 1;
  const double kc_w = a.ion.kc * a.w[i];
  float4* cur = (step & 1) ? a.posq1 : a.posq0;
  a.zq[i] = z1;
  a.qm[i] = static_cast<float>(z1 / a.mass[i]);
  cur[i].w = static_cast<float>(kc_w * z1);
  if (a.src_live) a.src_live[i / kLiveGroup] = 1;
  const uint4 wv = philox4x32_10(
      make_uint4(static_cast<uint32_t>(t), static_cast<uint32_t>(step),
                 static_cast<uint32_t>(static_cast<unsigned long long>(step) >> 32), 0u),
      make_uint2(static_cast<uint32_t>(a.ion.seed), static_cast<uint32_t>(a.ion.seed >> 32)));
  const double u1 = (static_cast<double>(wv.y) + 0.5) * (1.0 / 4294967296.0);
  const double u2 = (static_cast<double>(wv.z) + 0.5) * (1.0 / 4294967296.0);
  const double u3 = (static_cast<double>(wv.w) + 0.5) * (1.0 / 4294967296.0);
  const double ct = 2.0 * u1 - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
  const double ph = 2.0 * kPi * u2, rr = a.ion.r_create * cbrt(u3);
  const long long e = a.c.off + e_rel;
  const double X = a.x[i] + rr * st * cos(ph), Y = a.y[i] + rr * st * sin(ph), Z = a.z[i] + rr * ct;
  a.x[e] = X;
  a.y[e] = Y;
  a.z[e] = Z;
  a.ux[e] = a.ux[i];
  a.uy[e] = a.uy[i];
  a.uz[e] = a.uz[i];
  a.zq[e] = -1;
  a.qm[e] = -1.0f;
  a.w[e] = a.w[i];
  a.mass[e] = 1.0;
  a.kind[e] = 1;
  cur[e] = make_float4(static_cast<float>(X), static_cast<float>(Y), static_cast<float>(Z),
                       static_cast<float>(-kc_w));
  if (a.vel)
    a.vel[e] = make_float4(static_cast<float>(a.ux[i]), static_cast<float>(a.uy[i]),
                           static_cast<float>(a.uz[i]), static_cast<float>(a.w[i]));
  if (a.src_live) {
    a.src_live[e / kLiveGroup] = 1;
    a.tgt_live[e / kLiveGroup] = 1;
  }
}

// The fired ions, in index order, take the slots *pass_slot + (fired ions
// before them): each block adds the counts of the blocks before it (from
// k_ion_decide) to an in-block scan; the last block advances *next_slot.
__global__ void __launch_bounds__(256) k_ion_apply(const IonArgs a) {
  __shared__ int s_part[8], s_warp[8];
  __shared__ long long s_base;
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // fired ions of the blocks before this one
  int before = 0;
  for (int b = tid; b < static_cast<int>(blockIdx.x); b += 256) before += a.blk_fired[b];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) before += __shfl_xor_sync(0xffffffffu, before, d);
  if (lane == 0) s_part[warp] = before;
  const long long t = static_cast<long long>(blockIdx.x) * 256 + tid;
  const int f = (t < a.ion.n_ions) ? a.fired[t] : 0;
  const unsigned ball = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_warp[warp] = __popc(ball);
  __syncthreads();
  if (tid == 0) {
    long long b = 0;
    for (int w = 0; w < 8; ++w) b += s_part[w];
    s_base = *a.pass_slot + b;
  }
  __syncthreads();
  int wpre = 0, total = 0;
  for (int w = 0; w < 8; ++w) {
    wpre += (w < warp) ? s_warp[w] : 0;
    total += s_warp[w];
  }
  if (f) {
    const long long slot = s_base + wpre + __popc(ball & ((1u << lane) - 1u));
    // the upload check guarantees a free slot for every possible ionization
    if (MD_IN_RANGE(a.err, slot, a.ion.slot_base,
                    a.ion.slot_base + static_cast<long long>(a.ion.zmax) * a.ion.n_ions) &&
        MD_IN_RANGE(a.err, slot, 0, a.c.n)) {
      apply_one(a, step, t, slot);
      // the pass's charge changes in slot order, the sources of k_ion_fix: the
      // ion's extra charge at its position and its freed electron's record
      const long long k = slot - *a.pass_slot;
      if (a.fix_src && MD_IN_RANGE(a.err, k, 0, a.ion.n_ions)) {
        const float4* cur = (step & 1) ? a.posq1 : a.posq0;
        const float4 pi = cur[a.c.off + t];
        a.fix_src[k] = make_float4(pi.x, pi.y, pi.z,
                                   static_cast<float>(a.ion.kc) * static_cast<float>(a.w[a.c.off + t]));
        a.fix_src[a.ion.n_ions + k] = cur[a.c.off + slot];
      }
    }
  }
  if (blockIdx.x == gridDim.x - 1 && tid == 0) {
    const long long next = s_base + total;
    *a.next_slot = next;
    // the step splits the live records, below the new next free slot (with
    // the segment count the descriptor holds now)
    if (a.cl_dev)
      a.cl_dev->seg_len = live_seg_len(a.cl_dev->n_pad, a.cl_dev->nseg,
                                       next > a.ion.slot_base ? next : a.ion.slot_base);
  }
}

// Field at the ions after the pass's charge changes, for the step (clusters
// with a pass before every step).  The pass summed the field with the charges
// before its decisions; each ion j it fired gained one charge (K_C w_j) at x_j
// and freed an electron (charge -K_C w_j) at x_e.  By superposition the field
// the step would sum at ion t is e_ion[t] plus the field of those changes.
// k_ion_apply lists them as two source streams in slot order (fix_src: the
// ions' extra charges, then at n_ions the freed electrons), and k_ion_fix sums
// them at every ion with the step kernel's TMA-staged FP32/Kahan source loop:
// CTA (x, y) takes R x THREADS ions and segment y of the nf charge changes of
// each stream, and writes its partial field to scratch [seg][n_ions][3];
// k_ion_fix_combine adds the segments in order to e_ion (deterministic).
template <int THREADS, int R, int TILE, int STAGES, bool MI = false, bool PACK = false>
__global__ void __launch_bounds__(THREADS) k_ion_fix(const IonArgs a) {
  static_assert(!(PACK && MI), "minimum-image forces use the scalar path");
  __shared__ Stage<TILE, STAGES> sm;
  __shared__ DupTile<PACK ? TILE : 1> dup;
  __shared__ KahanSmem<PACK ? R / 2 : 1, PACK ? THREADS : 1, false> ks;
  __shared__ int s_abort;
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  const long long base = __ldcg(a.pass_slot);
  long long nf = __ldcg(a.next_slot) - base;
  nf = nf < 0 ? 0 : (nf > a.ion.n_ions ? a.ion.n_ions : nf);
  const long long per_seg = (nf + gridDim.y - 1) / gridDim.y;
  const long long j0 = static_cast<long long>(blockIdx.y) * per_seg;
  const long long jn = j0 >= nf ? 0 : (nf - j0 < per_seg ? nf - j0 : per_seg);
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  const long long t0 = static_cast<long long>(blockIdx.x) * (THREADS * R);
  float xi[R], yi[R], zi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = t0 + threadIdx.x + r * THREADS;
    const float4 p = (t < a.ion.n_ions) ? cur[a.c.off + t] : make_float4(0.f, 0.f, 0.f, 0.f);
    xi[r] = p.x;
    yi[r] = p.y;
    zi[r] = p.z;
  }
  Acc<R, false> acc;
  acc.zero();
  if constexpr (PACK) {
    // both halves of the changes into one set of Kahan sums (an empty
    // segment only clears them)
    unsigned it = 0;
    bool ok = true;
    for (int half = 0; half < 2 && ok; ++half)
      ok = sum_sources_packed<THREADS, R, TILE, STAGES, false>(
          sm, dup, ks, it, a.fix_src + half * a.ion.n_ions + j0, jn, xi, yi, zi, a.c.eps2, a.err,
          &s_abort, nullptr, 0, half == 0);
    if (!ok) return;
  } else if (jn > 0) {
    unsigned it = 0;
    bool ok = true;
    bool mi_on = false;
    if constexpr (MI) {
      const double t_n = a.c.t0 + static_cast<double>(step) * a.c.dt;
      mi_on = a.min_image && (a.c.boundary == 1 || (a.c.boundary == 2 && t_n < a.c.t_switch));
    }
    if (mi_on) {
      __shared__ float s_tb[6];
      target_bounds<THREADS, R>(xi, yi, zi, s_tb);
      const float L = static_cast<float>(a.c.box);
      for (int half = 0; half < 2 && ok; ++half)
        ok = sum_sources<THREADS, R, TILE, STAGES, false, true>(
            sm, it, a.fix_src + half * a.ion.n_ions + j0, jn, xi, yi, zi, a.c.eps2, acc, a.err,
            &s_abort, nullptr, 0, L, 1.0f / L, s_tb);
    } else {
      for (int half = 0; half < 2 && ok; ++half)
        ok = sum_sources<THREADS, R, TILE, STAGES, false>(
            sm, it, a.fix_src + half * a.ion.n_ions + j0, jn, xi, yi, zi, a.c.eps2, acc, a.err,
            &s_abort);
    }
    if (!ok) return;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long t = t0 + threadIdx.x + r * THREADS;
    if (t >= a.ion.n_ions) continue;
    if (!MD_IN_RANGE(a.err, blockIdx.y, 0, kIonMaxSeg)) continue;
    double* o = a.scratch + 3 * (static_cast<long long>(blockIdx.y) * a.ion.n_ions + t);
    if constexpr (PACK) {
      o[0] = -(static_cast<double>(kahan_part(ks, 0, r)) - kahan_part(ks, 3, r));
      o[1] = -(static_cast<double>(kahan_part(ks, 1, r)) - kahan_part(ks, 4, r));
      o[2] = -(static_cast<double>(kahan_part(ks, 2, r)) - kahan_part(ks, 5, r));
    } else {
      o[0] = -(static_cast<double>(acc.sx[r]) - acc.cx[r]);
      o[1] = -(static_cast<double>(acc.sy[r]) - acc.cy[r]);
      o[2] = -(static_cast<double>(acc.sz[r]) - acc.cz[r]);
    }
  }
}

// e_ion[t] += the charge-change field of k_ion_fix, its segments in order.
__global__ void __launch_bounds__(256) k_ion_fix_combine(const IonArgs a) {
  const long long step = __ldcg(a.step);
  if (!pass_active(a, step)) return;
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= a.ion.n_ions) return;
  double ex = 0.0, ey = 0.0, ez = 0.0;
  for (int sg = 0; sg < a.fix_nseg; ++sg) {
    const double* o = a.scratch + 3 * (static_cast<long long>(sg) * a.ion.n_ions + t);
    ex += o[0];
    ey += o[1];
    ez += o[2];
  }
  a.e_ion[3 * t + 0] += ex;
  a.e_ion[3 * t + 1] += ey;
  a.e_ion[3 * t + 2] += ez;
}

// Push of the first n_push ion records of cluster ci with the field of the
// pass (e_ion) instead of a direct sum: the step kernel's units skip the
// i-blocks that hold only these ions.  Runs after the pass and before the
// step kernel, which advances the step counter.
template <bool DET>
__global__ void __launch_bounds__(256) k_push_ions(const StepArgs a, int ci, const double* e_ion,
                                                  long long n_push) {
  __shared__ ClusterDev s_c;
  __shared__ float s_las[6];
  const long long step = __ldcg(a.step);
  if (threadIdx.x == 0) {
    s_c = a.cl[ci];
    laser_field(s_c, s_c.t0 + static_cast<double>(step) * s_c.dt, s_las);
  }
  __syncthreads();
  const long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_push) return;
  const float4* __restrict__ cur = (step & 1) ? a.posq1 : a.posq0;
  float4* __restrict__ nxt = (step & 1) ? a.posq0 : a.posq1;
  const double t_next = s_c.t0 + static_cast<double>(step + 1) * s_c.dt;
  push_record<DET>(a, s_c, s_c.off + t, e_ion[3 * t + 0], e_ion[3 * t + 1], e_ion[3 * t + 2],
                   s_las, t_next, cur, nxt);
}

// Liveness flags from the current records: a group of kLiveGroup records is
// a live source if one of them carries charge, a live target if one of them
// is not INACTIVE.
__global__ void k_live_init(const float4* posq0, const float4* posq1, const unsigned char* kind,
                            const long long* step, long long n_total, unsigned char* src_live,
                            unsigned char* tgt_live) {
  const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long r0 = g * kLiveGroup;
  if (r0 >= n_total) return;
  const float4* cur = (__ldcg(step) & 1) ? posq1 : posq0;
  const long long r1 = r0 + kLiveGroup < n_total ? r0 + kLiveGroup : n_total;
  unsigned char s = 0, t = 0;
  for (long long r = r0; r < r1; ++r) {
    if (cur[r].w != 0.0f) s = 1;
    if (kind[r] != 2) t = 1;
  }
  src_live[g] = s;
  tgt_live[g] = t;
}

constexpr int kIonThreads = 128;
constexpr int kIonR = 2;
constexpr int kIonTile = 512;
// the field pass without moments (cell-list moments): the step kernel's
// packed source loop
constexpr int kSumThreads = 128;
constexpr int kSumR = 8;
constexpr int kSumTile = 512;
constexpr bool kSumPacked = true;
// the charge-change field: the step kernel's packed source loop (eight
// targets per thread); the minimum-image twin is scalar (four per thread)
constexpr int kFixThreads = kIonThreads;
constexpr int kFixR = 8;
constexpr int kFixTile = 512;
constexpr int kFixMiR = 4;

}  // namespace

cudaError_t launch_live_init(const float4* posq0, const float4* posq1, const unsigned char* kind,
                             const long long* step, long long n_total, unsigned char* src_live,
                             unsigned char* tgt_live, cudaStream_t s) {
  const long long groups = (n_total + kLiveGroup - 1) / kLiveGroup;
  k_live_init<<<static_cast<unsigned>((groups + 255) / 256), 256, 0, s>>>(
      posq0, posq1, kind, step, n_total, src_live, tgt_live);
  return cudaGetLastError();
}

int ion_field_targets_per_cta() { return kIonThreads * kIonR; }

int ion_fix_targets_per_cta() { return kFixThreads * kFixR; }

int ion_sum_targets_per_cta() { return kSumThreads * kSumR; }

cudaError_t ion_sum_blocks_per_sm(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      out, k_ion_field_sum<kSumThreads, kSumR, kSumTile, 1, kSumPacked>, kSumThreads, 0);
}

cudaError_t ion_field_blocks_per_sm(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      out, k_ion_field<kIonThreads, kIonR, kIonTile, 2>, kIonThreads, 0);
}

cudaError_t ion_fix_blocks_per_sm(int* out) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      out, k_ion_fix<kFixThreads, kFixR, kFixTile, 1, false, true>, kFixThreads, 0);
}

cudaError_t launch_ion_pass(const IonArgs& a, cudaStream_t s) {
  if (a.ion.n_ions <= 0) return cudaSuccess;
  if (a.nseg < 1 || a.nseg > kIonMaxSeg) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (a.min_image || !a.cells.count) {
    // field and moments in one source loop
    const long long per = kIonThreads * kIonR;
    const dim3 g1(static_cast<unsigned>((a.ion.n_ions + per - 1) / per),
                  static_cast<unsigned>(a.nseg));
    if (a.min_image)
      k_ion_field<kIonThreads, kIonR, kIonTile, 2, true><<<g1, kIonThreads, 0, s>>>(a);
    else
      k_ion_field<kIonThreads, kIonR, kIonTile, 2><<<g1, kIonThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    // the field of the live records, then the moments from the cell list
    const long long per = kSumThreads * kSumR;
    const dim3 g1(static_cast<unsigned>((a.ion.n_ions + per - 1) / per),
                  static_cast<unsigned>(a.nseg));
    k_ion_field_sum<kSumThreads, kSumR, kSumTile, 1, kSumPacked><<<g1, kSumThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int cells = kCellBuckets;
    if ((e = cudaMemsetAsync(a.cells.count, 0, sizeof(int) * cells, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.cells.fill, 0, sizeof(int) * cells, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.cells.ion_count, 0, sizeof(int) * cells, s)) != cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(a.cells.ion_fill, 0, sizeof(int) * cells, s)) != cudaSuccess)
      return e;
    const unsigned gl = static_cast<unsigned>(std::min<long long>(4096, (a.c.n_pad + 255) / 256));
    const unsigned gi = static_cast<unsigned>(
        std::min<long long>(4096, (a.ion.n_ions + 255) / 256));
    k_cell_list<false><<<gl, 256, 0, s>>>(a);
    k_ion_cell_list<false><<<gi, 256, 0, s>>>(a);
    if ((e = launch_cell_scan(a, a.cells.count, a.cells.start, s)) != cudaSuccess) return e;
    if ((e = launch_cell_scan(a, a.cells.ion_count, a.cells.ion_start, s)) != cudaSuccess)
      return e;
    k_cell_list<true><<<gl, 256, 0, s>>>(a);
    k_ion_cell_list<true><<<gi, 256, 0, s>>>(a);
    k_ion_moments<<<static_cast<unsigned>((a.ion.n_ions + kMomIons - 1) / kMomIons),
                    kMomThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const unsigned g2 = static_cast<unsigned>((a.ion.n_ions + 255) / 256);
  k_ion_inputs<<<g2, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.ion.rate_model == 2 && a.mlp) {
    if ((e = launch_ion_mlp(a, s)) != cudaSuccess) return e;
  }
  k_ion_decide<<<g2, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ion_apply<<<g2, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.e_ion && a.fix_src) {
    if (a.fix_nseg < 1 || a.fix_nseg > kIonMaxSeg) return cudaErrorInvalidValue;
    const long long per_fix = kFixThreads * (a.min_image ? kFixMiR : kFixR);
    const dim3 gf(static_cast<unsigned>((a.ion.n_ions + per_fix - 1) / per_fix),
                  static_cast<unsigned>(a.fix_nseg));
    if (a.min_image)
      k_ion_fix<kFixThreads, kFixMiR, kFixTile, 2, true><<<gf, kFixThreads, 0, s>>>(a);
    else
      k_ion_fix<kFixThreads, kFixR, kFixTile, 1, false, true><<<gf, kFixThreads, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ion_fix_combine<<<g2, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_ion_push(const StepArgs& a, int ci, const double* e_ion, long long n_push,
                            bool det, cudaStream_t s) {
  if (n_push <= 0) return cudaSuccess;
  const unsigned g = static_cast<unsigned>((n_push + 255) / 256);
  if (det)
    k_push_ions<true><<<g, 256, 0, s>>>(a, ci, e_ion, n_push);
  else
    k_push_ions<false><<<g, 256, 0, s>>>(a, ci, e_ion, n_push);
  return cudaGetLastError();
}

}  // namespace md
