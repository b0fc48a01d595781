// md_runtime.cu -- host runtime behind the C ABI of include/md.h: context
// life cycle, device layout, graph-replayed stepping, autotuner, diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "md.h"
#include "md_internal.h"

namespace {

thread_local std::string g_last_error;

md_status fail(md_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

md_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(MD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(MD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MD_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr double kClassicalElectronRadius = 2.8179403262e-15;  // m, CODATA 2018
constexpr int kGraphSteps = 16;
constexpr double kMeC2Ev = 510998.95;  // electron rest energy, eV
// target slices start (and end, unless at the record count) on multiples of
// this, a multiple of every compiled i-block size, so that a slice is a whole
// number of i-blocks
constexpr int kSliceAlign = 1024;

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace

struct md_ctx {
  int device = 0;
  int sm_count = 0;
  int ion_field_bps = 1;   // resident CTAs per SM of the ionization field kernel
  int ion_fix_bps = 1;     // resident CTAs per SM of the charge-change field kernel
  int ion_sum_bps = 1;     // resident CTAs per SM of the field-only pass kernel
  int field_bps = 1;       // resident CTAs per SM of the field kernel (md_get_fields)
  double* d_field_part = nullptr;  // [kFieldMaxSeg][max n_pad][4] split partials
  double* d_diag_rec = nullptr;    // diagnostic steps: [n_total][6] per-record diagnostics
  double* d_part_phi = nullptr;    // diagnostic steps: [part_phi_seg][n_total] phi partials
  int part_phi_seg = 0;
  // per cluster: records live at the last upload (an ionizing cluster: below
  // its next free electron slot), for the choice of the source split
  std::vector<long long> live_host;
  // per cluster: the targets this context pushes, [slice_b, slice_e) of the
  // cluster's padded records (md_set_slice; default all of them)
  std::vector<long long> slice_b, slice_e;
  bool any_slice = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;

  int n_clusters = 0;
  std::vector<md::ClusterDev> cl;
  std::vector<double> kc;  // K_C of each cluster
  long long n_total = 0;   // padded records of all clusters
  long long max_n = 0;     // largest real record count of a cluster

  md::ClusterDev* d_cl = nullptr;
  float4* d_posq[2] = {nullptr, nullptr};
  double* d_x[3] = {nullptr, nullptr, nullptr};
  double* d_u[3] = {nullptr, nullptr, nullptr};
  float* d_qm = nullptr;
  double* d_w = nullptr;
  double* d_mass = nullptr;
  int* d_z = nullptr;
  unsigned char* d_kind = nullptr;
  long long* d_step = nullptr;
  unsigned* d_ticket = nullptr;
  unsigned* d_done = nullptr;
  int* d_err = nullptr;

  // field / diagnostics scratch (sized for the largest cluster)
  double* d_e = nullptr;
  double* d_phi = nullptr;
  md::DiagPartial* d_part = nullptr;
  md::DiagPartial* d_diag = nullptr;
  int diag_blocks = 0;

  // host <-> device staging for set/get (device raw buffer + pinned host)
  unsigned char* d_raw = nullptr;
  unsigned char* h_raw = nullptr;
  size_t raw_bytes = 0;
  md::DiagPartial* h_diag = nullptr;
  // one device word and its pinned host copy for synchronous queries: the
  // first record the upload check rejected (kNoBadRecord: none), the count
  // of active records
  unsigned long long* d_word = nullptr;
  unsigned long long* h_word = nullptr;

  // kernel configuration
  int cfg = -1;
  int ctas_per_sm = 0;
  int jsplit = 0;          // requested source segments (0: chosen by balance)
  int nseg_used = 1;       // largest segment count of any cluster
  md::Unit* d_units = nullptr;
  int n_units = 0;
  int* d_share_first = nullptr;  // first unit of every share, n_shares + 1
  int n_shares = 0;
  int grid = 0;
  double* d_fpart = nullptr;       // partial fields [nseg][n_total][3]
  size_t part_cap = 0;             // doubles allocated
  unsigned* d_iblk_cnt = nullptr;  // completion counter per i-block
  int iblk_cap = 0;

  cudaGraphExec_t graph = nullptr;

  // ionization
  std::vector<md::IonDev> ion;
  std::vector<long long> ion_out_off;  // per cluster, into d_ion_out / d_ion_fired
  bool any_ion = false;
  double* d_ion_scratch = nullptr;     // [kIonMaxSeg][max n_ions][kIonScratch]
  int* d_ion_blk = nullptr;            // [ceil(max n_ions / 256)] fired ions per block
  long long* d_ion_pass = nullptr;     // [n_clusters] first free slot at the pass start
  double* d_ion_out = nullptr;         // [sum n_ions][4]
  unsigned char* d_ion_fired = nullptr;
  double* d_ion_nu = nullptr;          // [sum n_ions] surrogate rates (-1: plain)
  // clusters with a pass before every step: the field at each ion after the
  // pass (the step pushes those ions with it) and the ions fired per pass
  double* d_ion_e = nullptr;           // [sum n_ions][3]
  float4* d_ion_fix = nullptr;         // [2 sum n_ions] charge changes of a pass (fix_src)
  // cell list of the local moments: ints (bounds, dims, grid, counts, starts,
  // fill counters) and the listed electrons' records, for the largest cluster
  int* d_cell_int = nullptr;
  float4* d_cell_rec = nullptr;
  long long cell_cap = 0;
  long long cell_ion_cap = 0;
  std::vector<long long> ion_push;     // per cluster: ion records pushed with d_ion_e
  unsigned char* d_src_live = nullptr; // liveness flags per kLiveGroup records
  unsigned char* d_tgt_live = nullptr;
  float4* d_vel = nullptr;             // FP32 (ux, uy, uz, w) per record
  long long* d_ion_next = nullptr;     // [n_clusters] next free electron slot

  // ion energy detectors (allocated by the first md_set_detectors)
  unsigned long long* d_det_hist = nullptr;  // [clusters][5][kDetMaxBins + 1]
  unsigned char* d_det_crossed = nullptr;    // [n_total]
  bool det_on = false;                       // some cluster has detectors
  // minimum-image forces: per-cluster flags (host and device), any set
  std::vector<unsigned char> min_image;
  unsigned char* d_min_image = nullptr;
  bool any_mi = false;
  float* d_mlp = nullptr;              // surrogate parameters (device), if set
};

constexpr int kDetMaxBins = 4096;  // energy bins per detector histogram

namespace {

size_t raw_record_bytes() {
  return 3 * sizeof(double) * 2 + sizeof(int) + 2 * sizeof(double) + 1;
}

// Host-layout staging: x[n][3], u[n][3], z[n], mass[n], w[n], kind[n].
struct RawView {
  double* x;
  double* u;
  int* z;
  double* mass;
  double* w;
  unsigned char* kind;
};

// Whether host memory is page-locked (registered or allocated by CUDA), so
// that an asynchronous copy can use it directly.
bool is_pinned(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

RawView raw_view(unsigned char* base, long long n) {
  RawView v;
  size_t o = 0;
  v.x = reinterpret_cast<double*>(base + o);
  o += sizeof(double) * 3 * n;
  v.u = reinterpret_cast<double*>(base + o);
  o += sizeof(double) * 3 * n;
  v.mass = reinterpret_cast<double*>(base + o);
  o += sizeof(double) * n;
  v.w = reinterpret_cast<double*>(base + o);
  o += sizeof(double) * n;
  v.z = reinterpret_cast<int*>(base + o);
  o += sizeof(int) * n;
  v.kind = base + o;
  return v;
}

md_status validate_config(const md_config& c, int idx) {
  if (!(c.dt > 0.0) || !std::isfinite(c.dt))
    return fail(MD_ERR_ARG, "cluster %d: dt must be > 0", idx);
  if (!(c.softening > 0.0) || !std::isfinite(c.softening) ||
      !(static_cast<float>(c.softening * c.softening) >= 1.1754944e-38f))
    return fail(MD_ERR_ARG,
                "cluster %d: softening must be > 0 with softening^2 a normal FP32 number (the "
                "GPU sum keeps the self pair)", idx);
  if (!std::isfinite(c.a0) || !std::isfinite(c.t0) || !std::isfinite(c.tau) ||
      !std::isfinite(c.box) || !std::isfinite(c.t_switch))
    return fail(MD_ERR_ARG, "cluster %d: a0, t0, tau, box and t_switch must be finite", idx);
  if (!(c.lambda_um > 0.0)) return fail(MD_ERR_ARG, "cluster %d: lambda_um must be > 0", idx);
  if (c.polarization != 0 && c.polarization != 1)
    return fail(MD_ERR_ARG, "cluster %d: polarization must be 0 or 1", idx);
  if (c.envelope < 0 || c.envelope > 3) return fail(MD_ERR_ARG, "cluster %d: bad envelope", idx);
  if (c.boundary < 0 || c.boundary > 2) return fail(MD_ERR_ARG, "cluster %d: bad boundary", idx);
  if (c.boundary != 0 && !(c.box > 0.0))
    return fail(MD_ERR_ARG, "cluster %d: periodic/mixed boundary needs box > 0", idx);
  if (c.envelope != MD_ENV_FLAT && !(c.tau > 0.0))
    return fail(MD_ERR_ARG, "cluster %d: tau must be > 0", idx);
  if (c.min_image != 0 && c.min_image != 1)
    return fail(MD_ERR_ARG, "cluster %d: min_image must be 0 or 1", idx);
  if (c.min_image && c.boundary == 0)
    return fail(MD_ERR_ARG, "cluster %d: min_image needs a periodic or mixed boundary", idx);
  if (c.rate_model < 0 || c.rate_model > 2)
    return fail(MD_ERR_ARG, "cluster %d: rate_model must be 0, 1 or 2", idx);
  return MD_OK;
}

// The ionization settings of a cluster of n records (rate_model != 0).
md_status validate_ionization_params(const md_config& c, long long n, int idx) {
  if (c.zmax < 1 || c.zmax > md::kMaxZ)
    return fail(MD_ERR_ARG, "cluster %d: zmax must be in [1, 16]", idx);
  if (c.n_ions < 1 || c.n_ions > n) return fail(MD_ERR_ARG, "cluster %d: bad n_ions", idx);
  if (c.slot_base < c.n_ions ||
      c.slot_base + static_cast<long long>(c.zmax) * c.n_ions > n)
    return fail(MD_ERR_ARG,
                "cluster %d: electron slots [slot_base, slot_base + zmax n_ions) must lie "
                "after the ions and inside the records", idx);
  if (c.ionize_every < 0) return fail(MD_ERR_ARG, "cluster %d: ionize_every < 0", idx);
  if (!(c.r_loc > 0.0) || !(c.r_create >= 0.0))
    return fail(MD_ERR_ARG, "cluster %d: r_loc must be > 0 and r_create >= 0", idx);
  for (int z = 0; z < c.zmax; ++z)
    if (!(c.ip_ev[z] > 0.0) || !(c.q_outer[z] >= 0.0))
      return fail(MD_ERR_ARG, "cluster %d: ip_ev[%d] must be > 0, q_outer >= 0", idx, z);
  return MD_OK;
}

md_status validate_ionization(const md_config& c, const md_particles& p, int idx) {
  if (c.rate_model == 0) return MD_OK;
  const md_status st = validate_ionization_params(c, p.n, idx);
  if (st != MD_OK) return st;
  for (long long i = 0; i < c.n_ions; ++i) {
    const int kd = p.kind ? p.kind[i] : (p.z[i] < 0 ? MD_KIND_ELECTRON : MD_KIND_ION);
    if (kd != MD_KIND_ION) return fail(MD_ERR_ARG, "cluster %d: record %lld < n_ions is not an ion", idx, i);
  }
  return MD_OK;
}

// The checks of one cluster's generation parameters and of its ionization
// settings against the generated record order.
md_status validate_generate(const md_config& c, const md_generate& g, int idx) {
  const bool fin = std::isfinite(g.r0) && std::isfinite(g.center[0]) &&
                   std::isfinite(g.center[1]) && std::isfinite(g.center[2]) &&
                   std::isfinite(g.ion_mass) && std::isfinite(g.weight) &&
                   std::isfinite(g.kt_e_ev) && std::isfinite(g.kt_i_ev);
  if (!fin) return fail(MD_ERR_ARG, "cluster %d: md_generate fields must be finite", idx);
  if (!(g.r0 > 0.0)) return fail(MD_ERR_ARG, "cluster %d: md_generate.r0 must be > 0", idx);
  if (!(g.ion_mass > 0.0))
    return fail(MD_ERR_ARG, "cluster %d: md_generate.ion_mass must be > 0", idx);
  if (!(g.weight > 0.0)) return fail(MD_ERR_ARG, "cluster %d: md_generate.weight must be > 0", idx);
  if (!(g.kt_e_ev >= 0.0) || !(g.kt_i_ev >= 0.0))
    return fail(MD_ERR_ARG, "cluster %d: md_generate temperatures must be >= 0", idx);
  if (g.n_ions < 0 || g.n_electrons < 0 || g.n_slots < 0)
    return fail(MD_ERR_ARG, "cluster %d: md_generate counts must be >= 0", idx);
  const long long n = static_cast<long long>(g.n_ions) + g.n_electrons + g.n_slots;
  if (n < 1 || n > (1LL << 30))
    return fail(MD_ERR_ARG, "cluster %d: md_generate record count must be in [1, 2^30]", idx);
  if (g.ion_charge < 0) return fail(MD_ERR_ARG, "cluster %d: md_generate.ion_charge < 0", idx);
  if (g.reserved != 0) return fail(MD_ERR_ARG, "cluster %d: md_generate.reserved must be 0", idx);
  if (c.rate_model == 0) return MD_OK;
  const md_status st = validate_ionization_params(c, n, idx);
  if (st != MD_OK) return st;
  if (c.n_ions > g.n_ions)
    return fail(MD_ERR_ARG, "cluster %d: n_ions = %d but only %lld records are ions", idx,
                c.n_ions, static_cast<long long>(g.n_ions));
  return MD_OK;
}

// The checks of one record (kind, mass, charge sign, finite x, u and w).
md_status check_record(const md_particles& p, int idx, long long i) {
  const int kd = p.kind ? p.kind[i] : (p.z[i] < 0 ? MD_KIND_ELECTRON : MD_KIND_ION);
  if (kd < 0 || kd > 2) return fail(MD_ERR_ARG, "cluster %d: record %lld: bad kind", idx, i);
  if (kd != MD_KIND_INACTIVE && !(p.mass[i] > 0.0))
    return fail(MD_ERR_ARG, "cluster %d: record %lld: mass must be > 0", idx, i);
  if (kd == MD_KIND_ELECTRON && p.z[i] >= 0)
    return fail(MD_ERR_ARG, "cluster %d: record %lld: electron with z >= 0", idx, i);
  if (kd == MD_KIND_ION && p.z[i] < 0)
    return fail(MD_ERR_ARG, "cluster %d: record %lld: ion with z < 0", idx, i);
  if (!(std::isfinite(p.x[3 * i]) && std::isfinite(p.x[3 * i + 1]) &&
        std::isfinite(p.x[3 * i + 2]) && std::isfinite(p.u[3 * i]) &&
        std::isfinite(p.u[3 * i + 1]) && std::isfinite(p.u[3 * i + 2]) &&
        std::isfinite(p.w[i])))
    return fail(MD_ERR_ARG, "cluster %d: record %lld: non-finite position, momentum or weight",
                idx, i);
  return MD_OK;
}

// Size and pointers of a particle block.
md_status check_block(const md_particles& p, int idx, long long expect_n) {
  if (p.n < 1) return fail(MD_ERR_ARG, "cluster %d: n must be >= 1", idx);
  if (expect_n >= 0 && p.n != expect_n)
    return fail(MD_ERR_ARG, "cluster %d: n = %lld, context holds %lld", idx, (long long)p.n,
                expect_n);
  if (p.n > (1LL << 30)) return fail(MD_ERR_ARG, "cluster %d: n too large", idx);
  if (!p.x || !p.u || !p.z || !p.mass || !p.w)
    return fail(MD_ERR_ARG, "cluster %d: x, u, z, mass and w are required", idx);
  return MD_OK;
}

md_status validate_particles(const md_particles& p, int idx, long long expect_n) {
  md_status st = check_block(p, idx, expect_n);
  if (st != MD_OK) return st;
  for (long long i = 0; i < p.n; ++i)
    if ((st = check_record(p, idx, i)) != MD_OK) return st;
  return MD_OK;
}

void destroy_graph(md_ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
}

md::StepArgs step_args(md_ctx* c) {
  md::StepArgs a;
  a.cl = c->d_cl;
  a.units = c->d_units;
  a.share_first = c->d_share_first;
  a.n_shares = c->n_shares;
  a.posq0 = c->d_posq[0];
  a.posq1 = c->d_posq[1];
  a.x = c->d_x[0];
  a.y = c->d_x[1];
  a.z = c->d_x[2];
  a.ux = c->d_u[0];
  a.uy = c->d_u[1];
  a.uz = c->d_u[2];
  a.qm = c->d_qm;
  a.step = c->d_step;
  a.ticket = c->d_ticket;
  a.done = c->d_done;
  a.err = c->d_err;
  a.part = c->d_fpart;
  a.iblk_cnt = c->d_iblk_cnt;
  a.n_total = c->n_total;
  a.src_live = c->d_src_live;
  a.tgt_live = c->d_tgt_live;
  a.vel = c->d_vel;
  a.det_hist = c->d_det_hist;
  a.det_crossed = c->d_det_crossed;
  a.mass = c->d_mass;
  a.diag_rec = nullptr;
  a.part_phi = nullptr;
  a.zq = c->d_z;
  a.kind = c->d_kind;
  a.w = c->d_w;
  a.min_image = c->d_min_image;
  return a;
}

// The step kernel a context with configuration k runs: the minimum-image
// twin when a cluster asks for image forces, the detector twin when a
// cluster has detectors, else the plain one.
cudaError_t launch_step_of(const md_ctx* c, const md::KernelConfig& k, const md::StepArgs& a,
                           cudaStream_t s) {
  if (c->any_mi) {
    if (!k.launch_step_mi) return cudaErrorInvalidValue;
    return c->det_on ? k.launch_step_mi_det(a, c->grid, s) : k.launch_step_mi(a, c->grid, s);
  }
  return c->det_on ? k.launch_step_det(a, c->grid, s) : k.launch_step(a, c->grid, s);
}

cudaError_t blocks_per_sm_of(const md_ctx* c, const md::KernelConfig& k, int* bps) {
  if (c->any_mi) {
    if (!k.max_blocks_per_sm_mi) return cudaErrorInvalidValue;
    return c->det_on ? k.max_blocks_per_sm_mi_det(bps) : k.max_blocks_per_sm_mi(bps);
  }
  return c->det_on ? k.max_blocks_per_sm_det(bps) : k.max_blocks_per_sm(bps);
}

// A cluster whose ionization pass runs before every step: the pass's field at
// its ions (corrected for the pass's own charge changes) is the step's field
// there, so the step pushes those ions with it instead of summing again.
bool ions_fused(const md_ctx* c, int ci) {
  const md::IonDev& io = c->ion[ci];
  return c->d_ion_e && io.rate_model != 0 && io.ionize_every == 1 && io.n_ions > 0;
}

// Cluster ci restricted to its target slice (the records md_diagnostics sums).
md::ClusterDev slice_view(const md_ctx* c, int ci) {
  md::ClusterDev v = c->cl[ci];
  const long long b = c->slice_b[ci], e = std::min<long long>(c->slice_e[ci], v.n);
  v.off += b;
  v.n = static_cast<int>(std::max(0LL, e - b));
  return v;
}

// Equal shares per resident CTA that md_autotune tries (jsplit = -k).
constexpr int kAutoShares[] = {2, 4};

// Source segments of md_get_fields / md_diagnostics at most.
constexpr int kFieldMaxSeg = 8;

// Segments per i-block for a requested split S: each segment holds at least
// one shared-memory tile of sources.
void segments_for(const md::ClusterDev& cl, int S, int tile, int* nseg, int* seg_len) {
  int n = std::max(1, std::min(S, cl.n_pad / tile));
  int len = (cl.n_pad + n - 1) / n;
  len = (len + md::kPad - 1) / md::kPad * md::kPad;
  *seg_len = len;
  *nseg = (cl.n_pad + len - 1) / len;
}

// Whether i-block b (of `per` targets) of cluster ci lies in the cluster's
// target slice (slice bounds are multiples of every i-block size).
bool block_in_slice(const md_ctx* c, int ci, long long b, long long per) {
  const long long i0 = b * per;
  return i0 >= c->slice_b[ci] && i0 < c->slice_e[ci];
}

long long units_for(const md_ctx* c, long long per, int S, int tile) {
  long long u = 0;
  for (int ci = 0; ci < c->n_clusters; ++ci) {
    const md::ClusterDev& cl = c->cl[ci];
    int ns, len;
    segments_for(cl, S, tile, &ns, &len);
    // i-blocks past the live records finish at once: count the live ones
    const long long live = ci < static_cast<int>(c->live_host.size()) ? c->live_host[ci] : cl.n_pad;
    const long long skip = ions_fused(c, ci) ? c->ion[ci].n_ions / per : 0;
    long long blocks = std::max(1LL, (std::max(1LL, live) + per - 1) / per - skip);
    if (c->slice_b[ci] > 0 || c->slice_e[ci] < cl.n_pad) {
      // a target slice: only its i-blocks
      const long long b0 = c->slice_b[ci] / per;
      const long long b1 = (std::min<long long>(c->slice_e[ci], cl.n_pad) + per - 1) / per;
      blocks = std::max(0LL, b1 - b0);
    }
    u += blocks * ns;
  }
  return std::max(1LL, u);
}

// Source split chosen for balance: equal units handed out by the ticket finish
// in ceil(units / slots) rounds; take the smallest split whose last round is
// at least 95 % full (or the best one up to 32).
int choose_split(const md_ctx* c, long long per, int tile, long long slots) {
  int best = 1;
  double best_eff = -1.0;
  for (int S = 1; S <= 32; ++S) {
    const long long u = units_for(c, per, S, tile);
    const long long rounds = (u + slots - 1) / slots;
    const double eff = static_cast<double>(u) / static_cast<double>(rounds * slots);
    if (eff >= 0.95) return S;
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = S;
    }
  }
  return best;
}

// Whether the step's source split must follow the live records, which only
// the device knows after each ionization pass (R16).
bool any_ionizing(const md_ctx* c) {
  for (int ci = 0; ci < c->n_clusters; ++ci)
    if (ci < static_cast<int>(c->ion.size()) && c->ion[ci].rate_model != 0) return true;
  return false;
}

// One pushed i-block for the share planner: its cluster, index in the
// cluster, index over all clusters, source tiles and the cluster's records.
struct BlockSpan {
  int ci, b, ib;
  long long tiles;
  int n_pad;
};

// Equal shares: the source tiles of the i-blocks `blks`, laid end to end (T
// tiles in all), are cut into G' = min(G, T) shares of floor or ceil of T / G'
// tiles, so the ticket's last round leaves no CTA idle.  A share is one or
// more pieces, each a tile range of one i-block's sources; the pieces of an
// i-block are numbered in source order.  Appends the units in share order and
// sets the first unit of every share (G' + 1 entries); returns G'.
long long plan_shares(const std::vector<BlockSpan>& blks, int tile, long long G,
                      std::vector<md::Unit>* units, std::vector<int>* first, int* max_parts) {
  long long T = 0;
  for (const BlockSpan& bk : blks) T += bk.tiles;
  G = std::max(1LL, std::min(G, T));
  auto bound = [&](long long k) { return k * T / G; };  // first tile of share k
  std::vector<int> share_of;
  long long F = 0, k = 0;
  *max_parts = 1;
  for (const BlockSpan& bk : blks) {
    const size_t u0 = units->size();
    for (long long p = F; p < F + bk.tiles;) {
      while (bound(k + 1) <= p) ++k;
      const long long q = std::min(F + bk.tiles, bound(k + 1));
      const long long j0 = (p - F) * tile;
      const long long j1 = std::min<long long>((q - F) * tile, bk.n_pad);
      md::Unit u{bk.ci, bk.b, static_cast<int>(units->size() - u0), bk.ib,
                 static_cast<int>(j0), static_cast<int>(j1 - j0), 0, 0};
      units->push_back(u);
      share_of.push_back(static_cast<int>(k));
      p = q;
    }
    const int np = static_cast<int>(units->size() - u0);
    for (size_t i = u0; i < units->size(); ++i) (*units)[i].nparts = np;
    *max_parts = std::max(*max_parts, np);
    F += bk.tiles;
  }
  first->assign(static_cast<size_t>(G) + 1, 0);
  for (int sh : share_of) ++(*first)[static_cast<size_t>(sh) + 1];
  for (size_t i = 1; i < first->size(); ++i) (*first)[i] += (*first)[i - 1];
  return G;
}

// Equal shares of a context's pushed i-blocks (those of its target slices)
// with G shares; the clusters' descriptors get one segment of all records.
void equal_shares(md_ctx* c, long long per, int tile, long long G, std::vector<md::Unit>* units,
                  std::vector<int>* first, int* max_parts) {
  std::vector<BlockSpan> blks;
  int ib = 0;
  for (int ci = 0; ci < c->n_clusters; ++ci) {
    md::ClusterDev& cl = c->cl[ci];
    cl.nseg = 1;
    cl.seg_len = cl.n_pad;
    c->ion_push[ci] = 0;
    const long long nb = (cl.n_pad + per - 1) / per;
    const long long tiles = std::max(1LL, (static_cast<long long>(cl.n_pad) + tile - 1) / tile);
    for (long long b = 0; b < nb; ++b, ++ib)
      if (block_in_slice(c, ci, b, per)) blks.push_back({ci, static_cast<int>(b), ib, tiles, cl.n_pad});
  }
  plan_shares(blks, tile, G, units, first, max_parts);
}

// Work units (cluster, i-block, source piece) and their shares.  jsplit < 0
// without ionizing clusters: equal shares, -jsplit per resident CTA.
// Otherwise every i-block's sources are split into segments (jsplit of them,
// or for 0 (and jsplit < 0 with ionizing clusters) a count chosen for
// balance) and the units, ordered by decreasing cost so the ticket hands the
// largest out first, are one share each.
md_status configure(md_ctx* c, int cfg, int ctas_per_sm, int jsplit) {
  int ncfg = 0;
  const md::KernelConfig* cfgs = md::step_configs(&ncfg);
  if (cfg < 0 || cfg >= ncfg) return fail(MD_ERR_ARG, "tuning index %d out of range", cfg);
  if (jsplit < -8 || jsplit > 64) return fail(MD_ERR_ARG, "jsplit must be in [-8, 64]");
  const md::KernelConfig& k = cfgs[cfg];
  const long long per = static_cast<long long>(k.threads) * k.r;
  if (c->any_mi && !k.launch_step_mi)
    return fail(MD_ERR_ARG, "configuration %d (packed) has no minimum-image kernel", cfg);
  int bps = 0;
  MD_CUDA(blocks_per_sm_of(c, k, &bps));
  if (bps < 1) return fail(MD_ERR_CUDA, "kernel configuration %d does not fit on an SM", cfg);
  const int cps = ctas_per_sm > 0 ? std::min(ctas_per_sm, bps) : bps;
  const long long slots = static_cast<long long>(cps) * c->sm_count;

  std::vector<md::Unit> units;
  std::vector<int> first;
  int ib = 0, max_seg = 1;
  const bool shares = jsplit < 0 && !any_ionizing(c);
  if (shares) {
    equal_shares(c, per, k.tile, slots * -jsplit, &units, &first, &max_seg);
    for (int ci = 0; ci < c->n_clusters; ++ci)
      ib += static_cast<int>((c->cl[ci].n_pad + per - 1) / per);
  } else {
    const int S = jsplit > 0 ? jsplit : choose_split(c, per, k.tile, slots);
    jsplit = std::max(jsplit, 0);
    struct Work {
      long long cost;
      md::Unit u;
    };
    std::vector<Work> work;
    for (int ci = 0; ci < c->n_clusters; ++ci) {
      md::ClusterDev& cl = c->cl[ci];
      segments_for(cl, S, k.tile, &cl.nseg, &cl.seg_len);
      max_seg = std::max(max_seg, cl.nseg);
      const long long nb = (cl.n_pad + per - 1) / per;
      // a cluster with a pass before every step: the i-blocks holding only
      // ions are pushed with the pass's field (launch_ion_push), not summed
      // again
      const long long skip = ions_fused(c, ci) ? c->ion[ci].n_ions / per : 0;
      c->ion_push[ci] = skip * per;
      for (long long b = 0; b < nb; ++b, ++ib) {
        if (b < skip || !block_in_slice(c, ci, b, per)) continue;
        for (int sg = 0; sg < cl.nseg; ++sg) {
          const long long len = std::min<long long>(cl.seg_len, cl.n_pad - static_cast<long long>(sg) * cl.seg_len);
          work.push_back({per * len, {ci, static_cast<int>(b), sg, ib, 0, -1, cl.nseg, 0}});
        }
      }
    }
    std::stable_sort(work.begin(), work.end(),
                     [](const Work& a, const Work& b) { return a.cost > b.cost; });
    units.reserve(work.size());
    for (auto& w : work) units.push_back(w.u);
    first.resize(units.size() + 1);
    for (size_t i = 0; i < first.size(); ++i) first[i] = static_cast<int>(i);
  }

  MD_CUDA(cudaStreamSynchronize(c->stream));
  if (c->d_units) cudaFree(c->d_units);
  c->d_units = nullptr;
  if (c->d_share_first) cudaFree(c->d_share_first);
  c->d_share_first = nullptr;
  MD_CUDA(dev_alloc(&c->d_units, units.size()));
  MD_CUDA(dev_alloc(&c->d_share_first, first.size()));
  MD_CUDA(cudaMemcpyAsync(c->d_units, units.data(), units.size() * sizeof(md::Unit),
                          cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaMemcpyAsync(c->d_share_first, first.data(), first.size() * sizeof(int),
                          cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaMemcpyAsync(c->d_cl, c->cl.data(), sizeof(md::ClusterDev) * c->n_clusters,
                          cudaMemcpyHostToDevice, c->stream));
  if (max_seg > 1) {
    const size_t need = static_cast<size_t>(max_seg) * static_cast<size_t>(c->n_total) * 3;
    if (need > c->part_cap) {
      cudaFree(c->d_fpart);
      c->d_fpart = nullptr;
      c->part_cap = 0;
      MD_CUDA(dev_alloc(&c->d_fpart, need));
      c->part_cap = need;
    }
    if (ib > c->iblk_cap) {
      cudaFree(c->d_iblk_cnt);
      c->d_iblk_cnt = nullptr;
      c->iblk_cap = 0;
      MD_CUDA(dev_alloc(&c->d_iblk_cnt, ib));
      c->iblk_cap = ib;
    }
    MD_CUDA(cudaMemsetAsync(c->d_iblk_cnt, 0, sizeof(unsigned) * ib, c->stream));
  }
  MD_CUDA(cudaStreamSynchronize(c->stream));
  c->n_units = static_cast<int>(units.size());
  c->n_shares = static_cast<int>(first.size() - 1);
  c->grid = static_cast<int>(std::max<long long>(1, std::min<long long>(c->n_shares, slots)));
  c->cfg = cfg;
  c->ctas_per_sm = ctas_per_sm;
  c->jsplit = jsplit;
  c->nseg_used = max_seg;
  destroy_graph(c);
  return MD_OK;
}

// Default before autotuning: 128 threads x 4 i-particles per thread, scalar.
int default_config(md_ctx* c) {
  (void)c;
  int ncfg = 0;
  const md::KernelConfig* cfgs = md::step_configs(&ncfg);
  for (int i = 0; i < ncfg; ++i)
    if (cfgs[i].threads == 128 && cfgs[i].r == 4 && !cfgs[i].packed) return i;
  return 0;
}

md_status ensure_scratch(md_ctx* c) {
  if (c->d_e) return MD_OK;
  MD_CUDA(dev_alloc(&c->d_field_part,
                    4 * static_cast<size_t>(kFieldMaxSeg) * static_cast<size_t>(c->max_n + md::kPad)));
  MD_CUDA(md::field_blocks_per_sm(&c->field_bps));
  MD_CUDA(dev_alloc(&c->d_e, 3 * static_cast<size_t>(c->max_n + md::kPad)));
  MD_CUDA(dev_alloc(&c->d_phi, static_cast<size_t>(c->max_n + md::kPad)));
  c->diag_blocks = std::max(1, std::min(4 * c->sm_count,
                                        static_cast<int>((c->max_n + md::kDiagThreads - 1) /
                                                         md::kDiagThreads)));
  MD_CUDA(dev_alloc(&c->d_part, c->diag_blocks));
  MD_CUDA(dev_alloc(&c->d_diag, 1));
  MD_CUDA(cudaMallocHost(reinterpret_cast<void**>(&c->h_diag), sizeof(md::DiagPartial)));
  return MD_OK;
}

md_status check_device_error(md_ctx* c) {
  int err = 0;
  MD_CUDA(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  if (err & md::kErrTimeout) {
    MD_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    MD_CUDA(cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), c->stream));
    MD_CUDA(cudaMemsetAsync(c->d_done, 0, sizeof(unsigned), c->stream));
    if (c->d_iblk_cnt)
      MD_CUDA(cudaMemsetAsync(c->d_iblk_cnt, 0, sizeof(unsigned) * c->iblk_cap, c->stream));
    return fail(MD_ERR_TIMEOUT, "a device-side wait exceeded its time budget");
  }
  if (err & md::kErrBounds) {
    MD_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    return fail(MD_ERR_STATE, "a device-side bounds check failed (checked build)");
  }
  return MD_OK;
}

md::IonArgs ion_args(md_ctx* c, int ci, int force) {
  md::IonArgs a;
  a.c = c->cl[ci];
  a.ion = c->ion[ci];
  a.posq0 = c->d_posq[0];
  a.posq1 = c->d_posq[1];
  a.x = c->d_x[0];
  a.y = c->d_x[1];
  a.z = c->d_x[2];
  a.ux = c->d_u[0];
  a.uy = c->d_u[1];
  a.uz = c->d_u[2];
  a.qm = c->d_qm;
  a.w = c->d_w;
  a.mass = c->d_mass;
  a.zq = c->d_z;
  a.kind = c->d_kind;
  a.step = c->d_step;
  a.err = c->d_err;
  a.force = force;
  a.scratch = c->d_ion_scratch;
  a.blk_fired = c->d_ion_blk;
  a.pass_slot = c->d_ion_pass + ci;
  // split the live sources of the field pass into nseg equal segments: the
  // (ion block, segment) CTAs fill whole waves of the resident CTA slots as
  // well as possible, with a small cost per extra segment; each segment keeps
  // at least 4 tiles of the cluster's records
  {
    // the field-only kernel when the moments come from the cell list
    const bool sum_only = !c->min_image[ci] && c->d_cell_int;
    const long long per = sum_only ? md::ion_sum_targets_per_cta() : md::ion_field_targets_per_cta();
    const long long ion_blocks = (a.ion.n_ions + per - 1) / per;
    const long long cap = std::max(1LL, static_cast<long long>(
        sum_only ? c->ion_sum_bps : c->ion_field_bps) * c->sm_count);
    const long long by_len = std::max(1LL, static_cast<long long>(a.c.n_pad) / 2048);
    const int smax = static_cast<int>(std::min<long long>(md::kIonMaxSeg, by_len));
    double best = -1.0;
    a.nseg = 1;
    for (int sg = 1; sg <= smax; ++sg) {
      const long long units = ion_blocks * sg;
      const long long waves = (units + cap - 1) / cap;
      const double score = static_cast<double>(units) / static_cast<double>(waves * cap) - 0.002 * sg;
      if (score > best + 1e-12) {
        best = score;
        a.nseg = sg;
      }
    }
  }
  a.out = c->d_ion_out + 4 * c->ion_out_off[ci];
  a.fired = c->d_ion_fired + c->ion_out_off[ci];
  a.nu = c->d_ion_nu + c->ion_out_off[ci];
  a.mlp = c->d_mlp;
  a.src_live = c->d_src_live;
  a.tgt_live = c->d_tgt_live;
  a.vel = c->d_vel;
  a.next_slot = c->d_ion_next + ci;
  a.cl_dev = c->d_cl + ci;
  a.min_image = c->min_image[ci];
  a.e_ion = ions_fused(c, ci) ? c->d_ion_e + 3 * c->ion_out_off[ci] : nullptr;
  a.fix_src = ions_fused(c, ci) ? c->d_ion_fix + 2 * c->ion_out_off[ci] : nullptr;
  std::memset(&a.cells, 0, sizeof(a.cells));
  if (!a.min_image && c->d_cell_int) {
    constexpr long long C = md::kCellBuckets;
    a.cells.count = c->d_cell_int + 16;
    a.cells.start = c->d_cell_int + 16 + C;
    a.cells.fill = c->d_cell_int + 16 + 2 * C + 1;
    a.cells.rec = c->d_cell_rec;
    a.cells.capacity = c->cell_cap;
    a.cells.ion_count = c->d_cell_int + 16 + 3 * C + 1;
    a.cells.ion_start = c->d_cell_int + 16 + 4 * C + 1;
    a.cells.ion_fill = c->d_cell_int + 16 + 5 * C + 2;
    a.cells.ion_list = c->d_cell_int + 16 + 6 * C + 2;
    a.cells.scan_tmp = c->d_cell_int + 16 + 6 * C + 2 + c->cell_ion_cap;
  }
  // segments of the charge-change field: about 3 waves of (ion block, segment) CTAs
  {
    const long long per = md::ion_fix_targets_per_cta();
    const long long blocks = std::max(1LL, (static_cast<long long>(a.ion.n_ions) + per - 1) / per);
    const long long cap = std::max(1LL, static_cast<long long>(c->ion_fix_bps) * c->sm_count);
    a.fix_nseg = static_cast<int>(std::max(1LL, std::min<long long>(
        md::kIonMaxSeg, (3 * cap + blocks - 1) / blocks)));
  }
  return a;
}

// Ionization passes of all clusters (the kernels skip themselves unless the
// device step is due or `force` is set).
cudaError_t launch_ion_all(md_ctx* c, int force, cudaStream_t s) {
  for (int ci = 0; ci < c->n_clusters; ++ci) {
    if (!c->ion[ci].rate_model) continue;
    if (!force && c->ion[ci].ionize_every <= 0) continue;
    cudaError_t e = md::launch_ion_pass(ion_args(c, ci, force), s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Pushes of the ions whose field the pass left (ions_fused), before the step
// kernel of the same step.
cudaError_t launch_ion_pushes(md_ctx* c, const md::StepArgs& a, cudaStream_t s) {
  for (int ci = 0; ci < c->n_clusters; ++ci) {
    if (!ions_fused(c, ci) || c->ion_push[ci] <= 0) continue;
    cudaError_t e = md::launch_ion_push(a, ci, c->d_ion_e + 3 * c->ion_out_off[ci],
                                        c->ion_push[ci], c->det_on, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

md_status launch_steps_direct(md_ctx* c, int n) {
  int ncfg = 0;
  const md::KernelConfig* cfgs = md::step_configs(&ncfg);
  const md::StepArgs a = step_args(c);
  for (int s = 0; s < n; ++s) {
    if (c->any_ion) {
      cudaError_t e = launch_ion_all(c, 0, c->stream);
      if (e == cudaSuccess) e = launch_ion_pushes(c, a, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "ionization launch");
    }
    cudaError_t e = launch_step_of(c, cfgs[c->cfg], a, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
  }
  return MD_OK;
}

md_status build_graph(md_ctx* c) {
  cudaStream_t cs = nullptr;
  MD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    int ncfg = 0;
    const md::KernelConfig* cfgs = md::step_configs(&ncfg);
    const md::StepArgs a = step_args(c);
    for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) {
      if (c->any_ion) e = launch_ion_all(c, 0, cs);
      if (c->any_ion && e == cudaSuccess) e = launch_ion_pushes(c, a, cs);
      if (e == cudaSuccess) e = launch_step_of(c, cfgs[c->cfg], a, cs);
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return cuda_fail(e, "capturing the step graph");
  }
  return MD_OK;
}

void free_ctx(md_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  cudaFree(c->d_cl);
  for (auto p : c->d_posq) cudaFree(p);
  for (auto p : c->d_x) cudaFree(p);
  for (auto p : c->d_u) cudaFree(p);
  cudaFree(c->d_qm);
  cudaFree(c->d_w);
  cudaFree(c->d_mass);
  cudaFree(c->d_z);
  cudaFree(c->d_kind);
  cudaFree(c->d_step);
  cudaFree(c->d_ticket);
  cudaFree(c->d_done);
  cudaFree(c->d_err);
  cudaFree(c->d_e);
  cudaFree(c->d_phi);
  cudaFree(c->d_part);
  cudaFree(c->d_diag);
  cudaFree(c->d_units);
  cudaFree(c->d_share_first);
  cudaFree(c->d_diag_rec);
  cudaFree(c->d_part_phi);
  cudaFree(c->d_min_image);
  cudaFree(c->d_field_part);
  cudaFree(c->d_fpart);
  cudaFree(c->d_iblk_cnt);
  cudaFree(c->d_raw);
  cudaFree(c->d_ion_scratch);
  cudaFree(c->d_ion_blk);
  cudaFree(c->d_ion_pass);
  cudaFree(c->d_ion_out);
  cudaFree(c->d_ion_fired);
  cudaFree(c->d_ion_nu);
  cudaFree(c->d_ion_e);
  cudaFree(c->d_ion_fix);
  cudaFree(c->d_cell_int);
  cudaFree(c->d_cell_rec);
  cudaFree(c->d_src_live);
  cudaFree(c->d_tgt_live);
  cudaFree(c->d_vel);
  cudaFree(c->d_ion_next);
  cudaFree(c->d_det_hist);
  cudaFree(c->d_det_crossed);
  cudaFree(c->d_mlp);
  if (c->h_raw) cudaFreeHost(c->h_raw);
  if (c->h_diag) cudaFreeHost(c->h_diag);
  cudaFree(c->d_word);
  if (c->h_word) cudaFreeHost(c->h_word);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

#define MD_STATUS(call)              \
  do {                               \
    const md_status s_ = (call);     \
    if (s_ != MD_OK) return s_;      \
  } while (0)

// Arguments of k_upload for n staged records (view d) of cluster ci.
md::UploadArgs upload_args(md_ctx* c, int ci, const RawView& d, long long n) {
  md::UploadArgs a;
  a.hx = d.x;
  a.hu = d.u;
  a.hz = d.z;
  a.hmass = d.mass;
  a.hw = d.w;
  a.hkind = d.kind;
  a.n = n;
  a.off = c->cl[ci].off;
  a.kc = c->kc[ci];
  a.posq0 = c->d_posq[0];
  a.posq1 = c->d_posq[1];
  a.x = c->d_x[0];
  a.y = c->d_x[1];
  a.z = c->d_x[2];
  a.ux = c->d_u[0];
  a.uy = c->d_u[1];
  a.uz = c->d_u[2];
  a.qm = c->d_qm;
  a.w = c->d_w;
  a.mass = c->d_mass;
  a.zq = c->d_z;
  a.kind = c->d_kind;
  a.step = c->d_step;
  a.vel = c->d_vel;
  a.first_bad = nullptr;
  return a;
}

md_status finish_upload(md_ctx* c, int ci, long long next_slot);

// Records of cluster ci from the caller's host arrays.  device_check: the
// records have not been checked on the host; k_validate checks the staged
// copy and a rejected block is not applied (clusters without ionization,
// whose upload has no other effect on the state).
md_status upload_cluster(md_ctx* c, int ci, const md_particles& p, bool device_check = false) {
  const long long n = p.n;
  long long next_slot = 0;
  if (c->d_ion_next && c->ion[ci].rate_model) {
    // electrons are freed into the slots after the last active one; all the
    // ionizations still possible must fit before the end of the slot region
    const md::IonDev& io = c->ion[ci];
    const long long end = io.slot_base + static_cast<long long>(io.zmax) * io.n_ions;
    long long last = -1, remaining = 0;
    for (long long r = io.slot_base; r < end; ++r) {
      const int kd = p.kind ? p.kind[r] : (p.z[r] < 0 ? MD_KIND_ELECTRON : MD_KIND_ION);
      if (kd != MD_KIND_INACTIVE) last = r;
    }
    for (long long i = 0; i < io.n_ions; ++i) remaining += std::max(0, io.zmax - p.z[i]);
    next_slot = last >= 0 ? last + 1 : io.slot_base;
    if (next_slot + remaining > end)
      return fail(MD_ERR_ARG,
                  "cluster %d: %lld more ionizations possible but only %lld free electron slots "
                  "after the last active one", ci, remaining, end - next_slot);
  }
  // each array goes to the device raw buffer directly when the caller's
  // memory is page-locked, else through the context's pinned staging buffer
  RawView h = raw_view(c->h_raw, n);
  RawView d = raw_view(c->d_raw, n);
  auto put = [&](void* dst, void* stage, const void* src, size_t bytes) -> cudaError_t {
    if (!is_pinned(src)) {
      std::memcpy(stage, src, bytes);
      src = stage;
    }
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
  };
  MD_CUDA(put(d.x, h.x, p.x, sizeof(double) * 3 * n));
  MD_CUDA(put(d.u, h.u, p.u, sizeof(double) * 3 * n));
  MD_CUDA(put(d.mass, h.mass, p.mass, sizeof(double) * n));
  MD_CUDA(put(d.w, h.w, p.w, sizeof(double) * n));
  MD_CUDA(put(d.z, h.z, p.z, sizeof(int) * n));
  if (p.kind) {
    MD_CUDA(put(d.kind, h.kind, p.kind, n));
  } else {
    for (long long i = 0; i < n; ++i)
      h.kind[i] = static_cast<unsigned char>(p.z[i] < 0 ? MD_KIND_ELECTRON : MD_KIND_ION);
    MD_CUDA(cudaMemcpyAsync(d.kind, h.kind, n, cudaMemcpyHostToDevice, c->stream));
  }
  md::UploadArgs a = upload_args(c, ci, d, n);
  a.first_bad = device_check ? c->d_word : nullptr;
  MD_CUDA(md::launch_upload(a, c->stream));
  if (device_check)
    MD_CUDA(cudaMemcpyAsync(c->h_word, c->d_word, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, c->stream));
  MD_STATUS(finish_upload(c, ci, next_slot));
  if (device_check && *c->h_word != md::kNoBadRecord) {
    // the message of the host check, for the first record the device rejected
    const md_status st = check_record(p, ci, static_cast<long long>(*c->h_word));
    return st != MD_OK ? st : fail(MD_ERR_ARG, "cluster %d: record %llu rejected", ci,
                                   *c->h_word);
  }
  return MD_OK;
}

// The state updates that follow an upload of cluster ci's records: its next
// free electron slot, the live records of the source split, the device
// descriptor's segment length and the liveness flags; then waits for the
// copies (the pinned staging buffer is reused by the next call).
md_status finish_upload(md_ctx* c, int ci, long long next_slot) {
  if (c->d_ion_next && c->ion[ci].rate_model)
    MD_CUDA(cudaMemcpyAsync(c->d_ion_next + ci, &next_slot, sizeof(long long),
                            cudaMemcpyHostToDevice, c->stream));
  if (static_cast<int>(c->live_host.size()) < c->n_clusters)
    c->live_host.resize(static_cast<size_t>(c->n_clusters), 0);
  c->live_host[ci] = (c->d_ion_next && c->ion[ci].rate_model) ? next_slot : c->cl[ci].n_pad;
  // the step's source segments must cover the new live records: reset the
  // device descriptor's segment length (once the split is configured)
  int live_len = 0;
  if (c->d_ion_next && c->ion[ci].rate_model && c->cl[ci].nseg >= 1) {
    live_len = md::live_seg_len(c->cl[ci].n_pad, c->cl[ci].nseg, next_slot);
    MD_CUDA(cudaMemcpyAsync(&c->d_cl[ci].seg_len, &live_len, sizeof(int), cudaMemcpyHostToDevice,
                            c->stream));
  }
  if (c->d_src_live)
    MD_CUDA(md::launch_live_init(c->d_posq[0], c->d_posq[1], c->d_kind, c->d_step, c->n_total,
                                 c->d_src_live, c->d_tgt_live, c->stream));
  // the pinned staging buffer is reused by the next call: wait for the copy
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return MD_OK;
}

// Records of cluster ci generated on the device (md_generate) into the
// staging buffer, then scattered into the state as an upload.
md_status generate_cluster(md_ctx* c, int ci, const md_generate& g) {
  const long long n = static_cast<long long>(g.n_ions) + g.n_electrons + g.n_slots;
  long long next_slot = 0;
  if (c->d_ion_next && c->ion[ci].rate_model) {
    // the active records are [0, n_ions + n_electrons); electrons are freed
    // into the slots after the last active one, and all the ionizations still
    // possible must fit before the end of the slot region
    const md::IonDev& io = c->ion[ci];
    const long long end = io.slot_base + static_cast<long long>(io.zmax) * io.n_ions;
    const long long n_act = static_cast<long long>(g.n_ions) + g.n_electrons;
    const long long last = io.slot_base < n_act ? std::min(end, n_act) - 1 : -1;
    const long long remaining =
        static_cast<long long>(io.n_ions) * std::max(0, io.zmax - g.ion_charge);
    next_slot = last >= 0 ? last + 1 : io.slot_base;
    if (next_slot + remaining > end)
      return fail(MD_ERR_ARG,
                  "cluster %d: %lld more ionizations possible but only %lld free electron slots "
                  "after the last active one", ci, remaining, end - next_slot);
  }
  RawView d = raw_view(c->d_raw, n);
  md::GenerateArgs ga;
  ga.r0 = g.r0;
  for (int k = 0; k < 3; ++k) ga.c[k] = g.center[k];
  ga.ion_mass = g.ion_mass;
  ga.weight = g.weight;
  ga.sig_i = g.kt_i_ev > 0.0 ? std::sqrt(g.kt_i_ev / (g.ion_mass * kMeC2Ev)) : 0.0;
  ga.sig_e = g.kt_e_ev > 0.0 ? std::sqrt(g.kt_e_ev / (1.0 * kMeC2Ev)) : 0.0;
  ga.n_ions = g.n_ions;
  ga.n_electrons = g.n_electrons;
  ga.n = n;
  ga.ion_charge = g.ion_charge;
  ga.seed = g.seed;
  ga.x = d.x;
  ga.u = d.u;
  ga.mass = d.mass;
  ga.w = d.w;
  ga.z = d.z;
  ga.kind = d.kind;
  MD_CUDA(md::launch_generate(ga, c->stream));
  md::UploadArgs a = upload_args(c, ci, d, n);
  a.first_bad = nullptr;
  MD_CUDA(md::launch_upload(a, c->stream));
  return finish_upload(c, ci, next_slot);
}

}  // namespace

namespace md {

md_status report_error(md_status status, const char* msg) { return fail(status, "%s", msg); }

md_status report_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

}  // namespace md

// ===================================================================== ABI

extern "C" {

const char* md_last_error(void) { return g_last_error.c_str(); }

double md_coulomb_constant(double lambda_um) {
  return 2.0 * kPi * kClassicalElectronRadius / (lambda_um * 1e-6);
}

double md_a0_from_intensity(double intensity_wcm2, double lambda_um) {
  return std::sqrt(intensity_wcm2 * lambda_um * lambda_um / 1.366e18);
}

double md_n_atoms(double r0, double r_wigner_seitz) {
  const double q = r0 / r_wigner_seitz;
  return q * q * q;
}

static md_status md_device_info_body(int32_t* sm_count, char* name, int32_t name_cap) {
  int dev = 0;
  MD_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  MD_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (sm_count) *sm_count = prop.multiProcessorCount;
  if (name && name_cap > 0) {
    std::strncpy(name, prop.name, name_cap - 1);
    name[name_cap - 1] = 0;
  }
  return MD_OK;
}

md_status md_device_info(int32_t* sm_count, char* name, int32_t name_cap) {
  return md::guarded([&] { return md_device_info_body(sm_count, name, name_cap); });
}

}  // extern "C"

namespace {

// A context for n_clusters clusters of nrec[i] records: device state
// allocated and zeroed (padding records INACTIVE at the origin), no records
// uploaded yet.  On failure nothing is left allocated.
md_status create_context(const md_config* cfgs, int32_t n_clusters, const long long* nrec,
                         void* stream, md_ctx** out) {
  md_ctx* c = new md_ctx();
  auto bail = [&](md_status st) {
    free_ctx(c);
    return st;
  };
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, c->device);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDeviceProperties"));
  if (prop.major != 10 || prop.minor != 3)
    return bail(fail(MD_ERR_UNSUPPORTED, "device %s is sm_%d%d; this library is built for sm_103a",
                     prop.name, prop.major, prop.minor));
  c->sm_count = prop.multiProcessorCount;
  e = md::ion_field_blocks_per_sm(&c->ion_field_bps);
  if (e == cudaSuccess) e = md::ion_fix_blocks_per_sm(&c->ion_fix_bps);
  if (e == cudaSuccess) e = md::ion_sum_blocks_per_sm(&c->ion_sum_bps);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor"));
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate"));
    c->own_stream = true;
  }

  c->n_clusters = n_clusters;
  long long off = 0;
  for (int i = 0; i < n_clusters; ++i) {
    const md_config& f = cfgs[i];
    md::ClusterDev d;
    std::memset(&d, 0, sizeof(d));  // detectors off
    d.off = off;
    d.n = static_cast<int>(nrec[i]);
    d.n_pad = static_cast<int>((nrec[i] + md::kPad - 1) / md::kPad * md::kPad);
    d.a0 = f.a0;
    d.tau = f.tau;
    d.t0 = f.t0;
    d.dt = f.dt;
    d.box = f.box;
    d.t_switch = f.t_switch;
    d.eps2 = static_cast<float>(f.softening * f.softening);
    d.pol = f.polarization;
    d.env = f.envelope;
    d.boundary = f.boundary;
    c->cl.push_back(d);
    c->kc.push_back(md_coulomb_constant(f.lambda_um));
    md::IonDev io;
    std::memset(&io, 0, sizeof(io));
    io.rate_model = f.rate_model;
    io.ionize_every = f.ionize_every;
    io.zmax = f.zmax;
    io.n_ions = f.rate_model ? f.n_ions : 0;
    io.slot_base = f.slot_base;
    io.seed = f.seed;
    io.r_loc = f.r_loc;
    io.r_create = f.r_create;
    io.kc = md_coulomb_constant(f.lambda_um);
    io.k_si = 2.0 * kPi / (f.lambda_um * 1e-6);
    io.omega = 299792458.0 * io.k_si;
    for (int z = 0; z < md::kMaxZ; ++z) {
      io.ip_ev[z] = f.ip_ev[z];
      io.q_outer[z] = f.q_outer[z];
    }
    c->ion_out_off.push_back(c->ion.empty() ? 0 : c->ion_out_off.back() + c->ion.back().n_ions);
    c->ion.push_back(io);
    c->ion_push.push_back(0);
    if (f.rate_model) c->any_ion = true;
    c->min_image.push_back(static_cast<unsigned char>(f.min_image));
    if (f.min_image) c->any_mi = true;
    c->slice_b.push_back(0);
    c->slice_e.push_back(d.n_pad);
    off += d.n_pad;
    c->max_n = std::max<long long>(c->max_n, nrec[i]);
  }
  c->n_total = off;
  const size_t N = static_cast<size_t>(c->n_total);

  md_status st = MD_OK;
#define MD_ALLOC(ptr, cnt)                                        \
  do {                                                            \
    cudaError_t e_ = dev_alloc(&(ptr), (cnt));                    \
    if (e_ != cudaSuccess) return bail(cuda_fail(e_, "cudaMalloc")); \
  } while (0)
  MD_ALLOC(c->d_cl, n_clusters);
  MD_ALLOC(c->d_posq[0], N);
  MD_ALLOC(c->d_posq[1], N);
  for (int k = 0; k < 3; ++k) {
    MD_ALLOC(c->d_x[k], N);
    MD_ALLOC(c->d_u[k], N);
  }
  MD_ALLOC(c->d_qm, N);
  MD_ALLOC(c->d_w, N);
  MD_ALLOC(c->d_mass, N);
  MD_ALLOC(c->d_z, N);
  MD_ALLOC(c->d_kind, N);
  MD_ALLOC(c->d_step, 1);
  MD_ALLOC(c->d_ticket, 1);
  MD_ALLOC(c->d_done, 1);
  MD_ALLOC(c->d_err, 1);
#undef MD_ALLOC
  c->raw_bytes = raw_record_bytes() * static_cast<size_t>(c->max_n) + 64;
  e = cudaMalloc(reinterpret_cast<void**>(&c->d_raw), c->raw_bytes);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
  e = cudaMallocHost(reinterpret_cast<void**>(&c->h_raw), c->raw_bytes);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMallocHost"));
  if (c->any_mi) {
    if (dev_alloc(&c->d_min_image, static_cast<size_t>(n_clusters)) != cudaSuccess)
      return bail(fail(MD_ERR_OOM, "minimum-image flags"));
    e = cudaMemcpy(c->d_min_image, c->min_image.data(), static_cast<size_t>(n_clusters),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMemcpy"));
  }
  if (dev_alloc(&c->d_word, 1) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&c->h_word), sizeof(unsigned long long)) !=
          cudaSuccess)
    return bail(fail(MD_ERR_OOM, "upload check buffers"));
  if (c->any_ion) {
    long long max_ion = 0, sum_ion = 0;
    for (auto& io : c->ion) {
      max_ion = std::max<long long>(max_ion, io.n_ions);
      sum_ion += io.n_ions;
    }
    if (dev_alloc(&c->d_ion_scratch, static_cast<size_t>(md::kIonMaxSeg) * md::kIonScratch *
                                         static_cast<size_t>(max_ion)) != cudaSuccess ||
        dev_alloc(&c->d_ion_blk, static_cast<size_t>((max_ion + 255) / 256)) != cudaSuccess ||
        dev_alloc(&c->d_ion_pass, static_cast<size_t>(n_clusters)) != cudaSuccess ||
        dev_alloc(&c->d_ion_out, 4 * static_cast<size_t>(sum_ion)) != cudaSuccess ||
        dev_alloc(&c->d_ion_fired, static_cast<size_t>(sum_ion)) != cudaSuccess ||
        dev_alloc(&c->d_ion_nu, static_cast<size_t>(sum_ion)) != cudaSuccess ||
        dev_alloc(&c->d_ion_e, 3 * static_cast<size_t>(sum_ion)) != cudaSuccess ||
        dev_alloc(&c->d_ion_fix, 2 * static_cast<size_t>(sum_ion)) != cudaSuccess)
      return bail(fail(MD_ERR_OOM, "ionization buffers"));
    const size_t groups = static_cast<size_t>((c->n_total + md::kLiveGroup - 1) / md::kLiveGroup);
    if (dev_alloc(&c->d_src_live, groups) != cudaSuccess ||
        dev_alloc(&c->d_tgt_live, groups) != cudaSuccess)
      return bail(fail(MD_ERR_OOM, "liveness flags"));
    if (dev_alloc(&c->d_vel, N) != cudaSuccess ||
        dev_alloc(&c->d_ion_next, static_cast<size_t>(n_clusters)) != cudaSuccess)
      return bail(fail(MD_ERR_OOM, "velocity stream"));
    {
      // cell list of the local moments, sized for the largest cluster
      constexpr size_t C = md::kCellBuckets;
      long long cap = 0;
      for (const auto& d : c->cl) cap = std::max<long long>(cap, d.n_pad);
      if (dev_alloc(&c->d_cell_int, 16 + 6 * C + 2 + static_cast<size_t>(max_ion) + C / 1024) !=
              cudaSuccess ||
          dev_alloc(&c->d_cell_rec, 2 * static_cast<size_t>(cap)) != cudaSuccess)
        return bail(fail(MD_ERR_OOM, "cell list"));
      c->cell_cap = cap;
      c->cell_ion_cap = max_ion;
    }
    cudaMemsetAsync(c->d_ion_next, 0, sizeof(long long) * n_clusters, c->stream);
    cudaMemsetAsync(c->d_vel, 0, N * sizeof(float4), c->stream);
    cudaMemsetAsync(c->d_ion_out, 0, sizeof(double) * 4 * sum_ion, c->stream);
    cudaMemsetAsync(c->d_ion_fired, 0, sum_ion, c->stream);
  }

  // zero state; padding records are INACTIVE with zero charge at the origin
  cudaStream_t s = c->stream;
  bool ok = true;
  ok &= cudaMemcpyAsync(c->d_cl, c->cl.data(), sizeof(md::ClusterDev) * n_clusters,
                        cudaMemcpyHostToDevice, s) == cudaSuccess;
  for (int k = 0; k < 2; ++k) ok &= cudaMemsetAsync(c->d_posq[k], 0, N * sizeof(float4), s) == cudaSuccess;
  for (int k = 0; k < 3; ++k) {
    ok &= cudaMemsetAsync(c->d_x[k], 0, N * sizeof(double), s) == cudaSuccess;
    ok &= cudaMemsetAsync(c->d_u[k], 0, N * sizeof(double), s) == cudaSuccess;
  }
  ok &= cudaMemsetAsync(c->d_qm, 0, N * sizeof(float), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_w, 0, N * sizeof(double), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_mass, 0, N * sizeof(double), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_z, 0, N * sizeof(int), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_kind, MD_KIND_INACTIVE, N, s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_step, 0, sizeof(long long), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_done, 0, sizeof(unsigned), s) == cudaSuccess;
  ok &= cudaMemsetAsync(c->d_err, 0, sizeof(int), s) == cudaSuccess;
  if (!ok) return bail(cuda_fail(cudaGetLastError(), "initialising device state"));
  (void)st;
  *out = c;
  return MD_OK;
}

// Records of every cluster in place (fill(c, i) uploads or generates cluster
// i), then the default kernel configuration.
template <class Fill>
md_status populate(md_ctx* c, int32_t n_clusters, Fill fill, md_ctx** out) {
  for (int i = 0; i < n_clusters; ++i) {
    const md_status st = fill(c, i);
    if (st != MD_OK) {
      free_ctx(c);
      return st;
    }
  }
  const md_status st = configure(c, default_config(c), 0, 0);
  if (st != MD_OK) {
    free_ctx(c);
    return st;
  }
  *out = c;
  return MD_OK;
}

}  // namespace

extern "C" {

static md_status md_init_body(md_ctx** out, const md_config* cfgs, int32_t n_clusters,
                              const md_particles* parts, void* stream) {
  if (!out) return fail(MD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_clusters < 1 || !cfgs || !parts) return fail(MD_ERR_ARG, "need >= 1 cluster");
  std::vector<long long> nrec(static_cast<size_t>(n_clusters));
  for (int i = 0; i < n_clusters; ++i) {
    md_status st = validate_config(cfgs[i], i);
    if (st != MD_OK) return st;
    st = validate_particles(parts[i], i, -1);
    if (st != MD_OK) return st;
    st = validate_ionization(cfgs[i], parts[i], i);
    if (st != MD_OK) return st;
    nrec[i] = parts[i].n;
  }
  md_ctx* c = nullptr;
  const md_status st = create_context(cfgs, n_clusters, nrec.data(), stream, &c);
  if (st != MD_OK) return st;
  return populate(c, n_clusters, [&](md_ctx* x, int i) { return upload_cluster(x, i, parts[i]); },
                  out);
}

md_status md_init(md_ctx** out, const md_config* cfgs, int32_t n_clusters,
                  const md_particles* parts, void* stream) {
  return md::guarded([&] { return md_init_body(out, cfgs, n_clusters, parts, stream); });
}

static md_status md_init_generate_body(md_ctx** out, const md_config* cfgs, const md_generate* gens,
                                       int32_t n_clusters, void* stream) {
  if (!out) return fail(MD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_clusters < 1 || !cfgs || !gens) return fail(MD_ERR_ARG, "need >= 1 cluster");
  std::vector<long long> nrec(static_cast<size_t>(n_clusters));
  for (int i = 0; i < n_clusters; ++i) {
    md_status st = validate_config(cfgs[i], i);
    if (st != MD_OK) return st;
    st = validate_generate(cfgs[i], gens[i], i);
    if (st != MD_OK) return st;
    nrec[i] = static_cast<long long>(gens[i].n_ions) + gens[i].n_electrons + gens[i].n_slots;
  }
  md_ctx* c = nullptr;
  const md_status st = create_context(cfgs, n_clusters, nrec.data(), stream, &c);
  if (st != MD_OK) return st;
  return populate(c, n_clusters, [&](md_ctx* x, int i) { return generate_cluster(x, i, gens[i]); },
                  out);
}

md_status md_init_generate(md_ctx** out, const md_config* cfgs, const md_generate* gens,
                           int32_t n_clusters, void* stream) {
  return md::guarded([&] { return md_init_generate_body(out, cfgs, gens, n_clusters, stream); });
}


void md_destroy(md_ctx* ctx) { free_ctx(ctx); }

static md_status md_step_body(md_ctx* c, int32_t nsteps) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (nsteps < 0) return fail(MD_ERR_ARG, "nsteps < 0");
  if (nsteps == 0) return MD_OK;
  if (nsteps >= kGraphSteps) {
    if (!c->graph) {
      md_status st = build_graph(c);
      if (st != MD_OK) return st;
    }
    for (int k = 0; k + kGraphSteps <= nsteps; k += kGraphSteps) {
      cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
  }
  return launch_steps_direct(c, nsteps % kGraphSteps);
}

md_status md_step(md_ctx* c, int32_t nsteps) {
  return md::guarded([&] { return md_step_body(c, nsteps); });
}

static md_status md_sync_body(md_ctx* c) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

md_status md_sync(md_ctx* c) {
  return md::guarded([&] { return md_sync_body(c); });
}

static md_status md_ionize_body(md_ctx* c) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (!c->any_ion) return MD_OK;
  cudaError_t e = launch_ion_all(c, 1, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ionization launch");
  return MD_OK;
}

md_status md_ionize(md_ctx* c) {
  return md::guarded([&] { return md_ionize_body(c); });
}

static md_status md_set_rate_mlp_body(md_ctx* c, const float* params, const md_mlp_train_config* domain) {
  if (!c || !params || !domain) return fail(MD_ERR_ARG, "NULL argument");
  if (!(domain->e_min > 0.0 && domain->e_max > domain->e_min && domain->ne_min > 0.0 &&
        domain->ne_max > domain->ne_min && domain->te_min > 0.0 &&
        domain->te_max > domain->te_min))
    return fail(MD_ERR_ARG, "bad surrogate domain");
  for (int ci = 0; ci < c->n_clusters; ++ci) {
    const md::IonDev& io = c->ion[ci];
    if (io.rate_model != 2) continue;
    if (io.zmax > 8)
      return fail(MD_ERR_ARG, "cluster %d: the surrogate has 8 outputs (zmax <= 8)", ci);
    // the surrogate's inputs are scaled by the species' ionization energies
    // and the laser wavelength it was trained for
    const double k_train = 2.0 * 3.14159265358979323846 / (domain->lambda_um * 1e-6);
    bool same = std::fabs(k_train - io.k_si) <= 1e-12 * io.k_si;
    for (int z = 0; z < io.zmax; ++z)
      same = same && std::fabs(domain->ip_ev[z] - io.ip_ev[z]) <= 1e-12 * io.ip_ev[z] &&
             domain->q_outer[z] == io.q_outer[z];
    if (!same)
      return fail(MD_ERR_ARG,
                  "cluster %d: the surrogate was trained for another species table or "
                  "wavelength", ci);
  }
  MD_CUDA(cudaStreamSynchronize(c->stream));
  if (!c->d_mlp) MD_CUDA(dev_alloc(&c->d_mlp, 5000));
  MD_CUDA(cudaMemcpyAsync(c->d_mlp, params, sizeof(float) * 5000, cudaMemcpyHostToDevice,
                          c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  for (auto& io : c->ion) {
    io.dom[0] = domain->e_min; io.dom[1] = domain->e_max;
    io.dom[2] = domain->ne_min; io.dom[3] = domain->ne_max;
    io.dom[4] = domain->te_min; io.dom[5] = domain->te_max;
  }
  destroy_graph(c);  // kernel arguments changed
  return MD_OK;
}

md_status md_set_rate_mlp(md_ctx* c, const float* params, const md_mlp_train_config* domain) {
  return md::guarded([&] { return md_set_rate_mlp_body(c, params, domain); });
}

static md_status md_set_detectors_body(md_ctx* c, int32_t cluster, const md_detector_config* d) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  if (d && !(d->radius > 0.0 && d->cone_half_angle_deg >= 0.0 &&
             d->cone_half_angle_deg <= 90.0 && d->e_max_ev > 0.0 && d->n_bins >= 1 &&
             d->n_bins <= kDetMaxBins && d->reserved == 0 && std::isfinite(d->center[0]) &&
             std::isfinite(d->center[1]) && std::isfinite(d->center[2])))
    return fail(MD_ERR_ARG, "detectors: radius > 0, cone in [0, 90] degrees, e_max_ev > 0, "
                "1 <= n_bins <= %d, reserved = 0, finite centre", kDetMaxBins);
  if (d && c->any_slice)
    return fail(MD_ERR_STATE, "detectors are not available in a context with target slices");
  MD_CUDA(cudaStreamSynchronize(c->stream));
  const size_t per = 5 * static_cast<size_t>(kDetMaxBins + 1);
  if (d && !c->d_det_hist) {
    MD_CUDA(dev_alloc(&c->d_det_hist, per * c->n_clusters));
    MD_CUDA(dev_alloc(&c->d_det_crossed, static_cast<size_t>(c->n_total)));
    MD_CUDA(cudaMemsetAsync(c->d_det_hist, 0, sizeof(unsigned long long) * per * c->n_clusters,
                            c->stream));
    MD_CUDA(cudaMemsetAsync(c->d_det_crossed, 0, static_cast<size_t>(c->n_total), c->stream));
  }
  md::ClusterDev& cl = c->cl[cluster];
  if (d) {
    cl.det_nbins = d->n_bins;
    cl.det_r2 = d->radius * d->radius;
    cl.det_cos = std::cos(d->cone_half_angle_deg * 3.14159265358979323846 / 180.0);
    cl.det_emax = d->e_max_ev;
    for (int k = 0; k < 3; ++k) cl.det_c[k] = d->center[k];
    cl.det_off = static_cast<long long>(per) * cluster;
    // a new configuration starts empty
    MD_CUDA(cudaMemsetAsync(c->d_det_hist + per * cluster, 0, sizeof(unsigned long long) * per,
                            c->stream));
    MD_CUDA(cudaMemsetAsync(c->d_det_crossed + cl.off, 0, static_cast<size_t>(cl.n_pad),
                            c->stream));
  } else {
    cl.det_nbins = 0;
  }
  MD_CUDA(cudaMemcpyAsync(c->d_cl + cluster, &cl, sizeof(md::ClusterDev),
                          cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  destroy_graph(c);  // kernel arguments changed
  bool on = false;
  for (const auto& k : c->cl) on = on || k.det_nbins > 0;
  if (on != c->det_on) {
    // the step kernels with and without the detector epilogue are separate
    // instantiations (possibly with other occupancy): size the grid anew
    c->det_on = on;
    md_status st = configure(c, c->cfg, c->ctas_per_sm, c->jsplit);
    if (st != MD_OK) return st;
  }
  return check_device_error(c);
}

md_status md_set_detectors(md_ctx* c, int32_t cluster, const md_detector_config* d) {
  return md::guarded([&] { return md_set_detectors_body(c, cluster, d); });
}

static md_status md_get_iedf_body(md_ctx* c, int32_t cluster, uint64_t* detected, uint64_t* inside) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  const md::ClusterDev& cl = c->cl[cluster];
  if (!c->d_det_hist || cl.det_nbins <= 0)
    return fail(MD_ERR_STATE, "cluster %d has no detectors (md_set_detectors)", cluster);
  const int nb1 = cl.det_nbins + 1;
  std::vector<unsigned long long> h(5 * static_cast<size_t>(nb1));
  MD_CUDA(cudaMemcpyAsync(h.data(), c->d_det_hist + cl.det_off,
                          sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost,
                          c->stream));
  std::vector<unsigned long long> hin;
  if (inside) {
    unsigned long long* d_in = nullptr;
    MD_CUDA(dev_alloc(&d_in, static_cast<size_t>(nb1)));
    cudaError_t e = cudaMemsetAsync(d_in, 0, sizeof(unsigned long long) * nb1, c->stream);
    if (e == cudaSuccess)
      e = md::launch_iedf_inside(cl, c->d_u[0], c->d_u[1], c->d_u[2], c->d_mass, c->d_z,
                                 c->d_kind, c->d_det_crossed, d_in, c->stream);
    hin.resize(nb1);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hin.data(), d_in, sizeof(unsigned long long) * nb1,
                          cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_in);
    if (e != cudaSuccess) return cuda_fail(e, "inside IEDF");
  }
  MD_CUDA(cudaStreamSynchronize(c->stream));
  if (detected)
    for (size_t k = 0; k < h.size(); ++k) detected[k] = h[k];
  if (inside)
    for (int k = 0; k < nb1; ++k) inside[k] = hin[k];
  return check_device_error(c);
}

md_status md_get_iedf(md_ctx* c, int32_t cluster, uint64_t* detected, uint64_t* inside) {
  return md::guarded([&] { return md_get_iedf_body(c, cluster, detected, inside); });
}

static md_status md_get_ionization_body(md_ctx* c, int32_t cluster, double* emag, double* ne, double* te,
                                        double* prob, uint8_t* fired) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  const long long n = c->ion[cluster].n_ions;
  if (!c->ion[cluster].rate_model || n == 0) return fail(MD_ERR_STATE, "cluster has no ionization");
  std::vector<double> out(4 * n);
  MD_CUDA(cudaMemcpyAsync(out.data(), c->d_ion_out + 4 * c->ion_out_off[cluster],
                          sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, c->stream));
  if (fired)
    MD_CUDA(cudaMemcpyAsync(fired, c->d_ion_fired + c->ion_out_off[cluster], n,
                            cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  for (long long i = 0; i < n; ++i) {
    if (emag) emag[i] = out[4 * i];
    if (ne) ne[i] = out[4 * i + 1];
    if (te) te[i] = out[4 * i + 2];
    if (prob) prob[i] = out[4 * i + 3];
  }
  return check_device_error(c);
}

md_status md_get_ionization(md_ctx* c, int32_t cluster, double* emag, double* ne, double* te,
                            double* prob, uint8_t* fired) {
  return md::guarded([&] { return md_get_ionization_body(c, cluster, emag, ne, te, prob, fired); });
}

static md_status md_set_step_body(md_ctx* c, int64_t step) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (step < 0) return fail(MD_ERR_ARG, "step < 0");
  // the j-stream buffer in use is selected by the parity of the step: move
  // the current positions to the buffer of the new parity
  long long cur = 0;
  MD_CUDA(cudaMemcpyAsync(&cur, c->d_step, sizeof(cur), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  if ((cur & 1) != (step & 1))
    MD_CUDA(cudaMemcpyAsync(c->d_posq[step & 1], c->d_posq[cur & 1],
                            sizeof(float4) * static_cast<size_t>(c->n_total),
                            cudaMemcpyDeviceToDevice, c->stream));
  long long v = step;
  MD_CUDA(cudaMemcpyAsync(c->d_step, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return MD_OK;
}

md_status md_set_step(md_ctx* c, int64_t step) {
  return md::guarded([&] { return md_set_step_body(c, step); });
}

static md_status md_wait_selftest_body(md_ctx* c, double budget_ms) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (!(budget_ms > 0.0) || budget_ms > 5000.0)
    return fail(MD_ERR_ARG, "budget_ms must be in (0, 5000]");
  int clk_khz = 0;
  MD_CUDA(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, c->device));
  const long long budget = static_cast<long long>(budget_ms * clk_khz);
  MD_CUDA(md::launch_wait_selftest(budget, c->d_err, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

md_status md_wait_selftest(md_ctx* c, double budget_ms) {
  return md::guarded([&] { return md_wait_selftest_body(c, budget_ms); });
}

static md_status md_set_slice_body(md_ctx* c, int32_t cluster, int64_t i_begin, int64_t i_end) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  const md::ClusterDev& cl = c->cl[cluster];
  if (i_begin < 0 || i_end < i_begin || i_end > cl.n)
    return fail(MD_ERR_ARG, "slice [%lld, %lld) must lie in [0, %d]", (long long)i_begin,
                (long long)i_end, cl.n);
  if ((i_begin % kSliceAlign != 0 && i_begin != cl.n) ||
      (i_end % kSliceAlign != 0 && i_end != cl.n))
    return fail(MD_ERR_ARG, "slice bounds must be multiples of %d (or the record count)",
                kSliceAlign);
  if (c->any_ion || c->det_on)
    return fail(MD_ERR_STATE, "target slices need a context without ionization or detectors");
  MD_CUDA(cudaStreamSynchronize(c->stream));
  c->slice_b[cluster] = i_begin;
  c->slice_e[cluster] = i_end == cl.n ? cl.n_pad : i_end;
  bool any = false;
  for (int ci = 0; ci < c->n_clusters; ++ci)
    any = any || c->slice_b[ci] > 0 || c->slice_e[ci] < c->cl[ci].n_pad;
  c->any_slice = any;
  return configure(c, c->cfg, c->ctas_per_sm, c->jsplit);
}

md_status md_set_slice(md_ctx* c, int32_t cluster, int64_t i_begin, int64_t i_end) {
  return md::guarded([&] { return md_set_slice_body(c, cluster, i_begin, i_end); });
}

static md_status md_get_jstream_body(md_ctx* c, int32_t cluster, void** posq, int64_t* n_pad) {
  if (!c || !posq || !n_pad) return fail(MD_ERR_ARG, "NULL argument");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  long long step = 0;
  MD_CUDA(cudaMemcpyAsync(&step, c->d_step, sizeof(step), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  *posq = static_cast<void*>(c->d_posq[step & 1] + c->cl[cluster].off);
  *n_pad = c->cl[cluster].n_pad;
  return check_device_error(c);
}

md_status md_get_jstream(md_ctx* c, int32_t cluster, void** posq, int64_t* n_pad) {
  return md::guarded([&] { return md_get_jstream_body(c, cluster, posq, n_pad); });
}

static md_status md_get_step_body(md_ctx* c, int64_t* step) {
  if (!c || !step) return fail(MD_ERR_ARG, "NULL argument");
  long long v = 0;
  MD_CUDA(cudaMemcpyAsync(&v, c->d_step, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  *step = v;
  return MD_OK;
}

md_status md_get_step(md_ctx* c, int64_t* step) {
  return md::guarded([&] { return md_get_step_body(c, step); });
}

static md_status run_fields(md_ctx* c, int ci, bool potential) {
  md_status st = ensure_scratch(c);
  if (st != MD_OK) return st;
  long long step = 0;
  MD_CUDA(cudaMemcpyAsync(&step, c->d_step, sizeof(step), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  const md::ClusterDev& cl = c->cl[ci];
  const float4* cur = c->d_posq[step & 1] + cl.off;
  // targets: the cluster's slice (all its records unless md_set_slice)
  const long long sb = c->slice_b[ci], se = std::min<long long>(c->slice_e[ci], cl.n_pad);
  md::FieldArgs a;
  a.src = cur;
  a.ns = cl.n_pad;
  a.tgt = cur + sb;
  a.nt = std::max(0LL, se - sb);
  a.eps2 = cl.eps2;
  a.self_offset = sb;
  a.e = c->d_e;
  a.phi = potential ? c->d_phi : nullptr;
  a.err = c->d_err;
  a.src_live = c->d_src_live;
  a.tgt_live = c->d_tgt_live;
  a.gbase = cl.off;
  // minimum-image displacements while this cluster's boundary is periodic
  const double t_n = cl.t0 + static_cast<double>(step) * cl.dt;
  if (c->min_image[ci] && (cl.boundary == 1 || (cl.boundary == 2 && t_n < cl.t_switch)))
    a.box = static_cast<float>(cl.box);
  // split the sources so that about 4 waves of CTAs run (at most kFieldMaxSeg
  // segments of at least 4 tiles each)
  const long long per = md::field_targets_per_cta();
  const long long blocks = (a.nt + per - 1) / per;
  const long long want = (4LL * c->field_bps * c->sm_count + blocks - 1) / blocks;
  const long long nseg = std::max(1LL, std::min({want, static_cast<long long>(kFieldMaxSeg),
                                                a.ns / 2048}));
  if (nseg > 1) {
    a.nseg = static_cast<int>(nseg);
    a.seg_len = (a.ns + nseg - 1) / nseg;
    a.part = c->d_field_part;
  }
  MD_CUDA(md::launch_field(a, potential, c->stream));
  return MD_OK;
}

static md_status md_get_fields_body(md_ctx* c, int32_t cluster, double* e, double* phi) {
  if (!c || !e) return fail(MD_ERR_ARG, "NULL argument");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  md_status st = run_fields(c, cluster, phi != nullptr);
  if (st != MD_OK) return st;
  // the records of the cluster's target slice (all of them unless md_set_slice)
  const long long sb = c->slice_b[cluster];
  const long long n = std::max(0LL, std::min<long long>(c->slice_e[cluster], c->cl[cluster].n) - sb);
  MD_CUDA(cudaMemcpyAsync(e + 3 * sb, c->d_e, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                          c->stream));
  if (phi)
    MD_CUDA(cudaMemcpyAsync(phi + sb, c->d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost,
                            c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

md_status md_get_fields(md_ctx* c, int32_t cluster, double* e, double* phi) {
  return md::guarded([&] { return md_get_fields_body(c, cluster, e, phi); });
}

static md_status md_count_active_body(md_ctx* c, int32_t cluster, int64_t* out) {
  if (!c || !out) return fail(MD_ERR_ARG, "NULL argument");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  MD_CUDA(md::launch_count_active(c->d_kind, c->cl[cluster].off, c->cl[cluster].n,
                                  c->d_word, c->stream));
  MD_CUDA(cudaMemcpyAsync(c->h_word, c->d_word, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  md_status st = check_device_error(c);
  if (st != MD_OK) return st;
  *out = static_cast<int64_t>(*c->h_word);
  return MD_OK;
}

md_status md_count_active(md_ctx* c, int32_t cluster, int64_t* out) {
  return md::guarded([&] { return md_count_active_body(c, cluster, out); });
}

// md_diag of a cluster from its reduced partials, at step `step`.
md_status fill_diag(const md::DiagPartial& d, long long step, const md::ClusterDev& cl,
                    md_diag* out) {
  std::memset(out, 0, sizeof(*out));
  out->step = step;
  out->t = cl.t0 + static_cast<double>(step) * cl.dt;
  out->ke = d.v[0];
  out->ke_ions = d.v[1];
  out->ke_electrons = d.v[2];
  out->pe = d.v[3];
  out->total = d.v[0] + d.v[3];
  out->p[0] = d.v[4];
  out->p[1] = d.v[5];
  out->p[2] = d.v[6];
  out->n_active = d.cnt[0];
  out->n_nonfinite = d.cnt[1];
  for (int k = 0; k < md::kHistBins; ++k) {
    out->charge_count[k] = d.hist[k];
    out->charge_weight[k] = d.histw[k];
  }
  if (out->n_nonfinite > 0)
    return fail(MD_ERR_NONFINITE, "%lld records hold NaN/Inf", (long long)out->n_nonfinite);
  return MD_OK;
}

static md_status md_diagnostics_body(md_ctx* c, int32_t cluster, md_diag* out) {
  if (!c || !out) return fail(MD_ERR_ARG, "NULL argument");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  md_status st = run_fields(c, cluster, true);
  if (st != MD_OK) return st;
  md::DiagArgs a;
  a.c = slice_view(c, cluster);
  a.x = c->d_x[0];
  a.y = c->d_x[1];
  a.z = c->d_x[2];
  a.ux = c->d_u[0];
  a.uy = c->d_u[1];
  a.uz = c->d_u[2];
  a.qm = c->d_qm;
  a.w = c->d_w;
  a.mass = c->d_mass;
  a.zq = c->d_z;
  a.kind = c->d_kind;
  a.e = c->d_e;
  a.phi = c->d_phi;
  a.step = c->d_step;
  a.part = c->d_part;
  MD_CUDA(md::launch_diag(a, c->diag_blocks, c->d_diag, c->stream));
  MD_CUDA(cudaMemcpyAsync(c->h_diag, c->d_diag, sizeof(md::DiagPartial), cudaMemcpyDeviceToHost,
                          c->stream));
  long long step = 0;
  MD_CUDA(cudaMemcpyAsync(&step, c->d_step, sizeof(step), cudaMemcpyDeviceToHost, c->stream));
  MD_CUDA(cudaStreamSynchronize(c->stream));
  st = check_device_error(c);
  if (st != MD_OK) return st;
  return fill_diag(*c->h_diag, step, a.c, out);
}

md_status md_diagnostics(md_ctx* c, int32_t cluster, md_diag* out) {
  return md::guarded([&] { return md_diagnostics_body(c, cluster, out); });
}

// One step of every cluster that also reports each cluster's diagnostics at
// the start of the step: the step kernel's POT twin sums the potential beside
// the field and records every record's diagnostics from its own kick, and an
// O(N) reduction per cluster adds them in a fixed order.  Contexts with
// ionization, detectors or minimum-image forces take the diagnostics call
// and md_step(1) instead.
static md_status md_step_diag_body(md_ctx* c, md_diag* out) {
  if (!c || !out) return fail(MD_ERR_ARG, "NULL argument");
  int ncfg = 0;
  const md::KernelConfig* cfgs = md::step_configs(&ncfg);
  const md::KernelConfig& k = cfgs[c->cfg];
  md_status st = MD_OK, worst = MD_OK;
  if (c->any_ion || c->det_on || c->any_mi || !k.launch_step_pot) {
    for (int ci = 0; ci < c->n_clusters; ++ci) {
      st = md_diagnostics(c, ci, &out[ci]);
      if (st == MD_ERR_NONFINITE) worst = st;
      else if (st != MD_OK) return st;
    }
    st = md_step(c, 1);
    return st != MD_OK ? st : (worst != MD_OK ? fail(worst, "records hold NaN/Inf") : MD_OK);
  }
  st = ensure_scratch(c);
  if (st != MD_OK) return st;
  const size_t nt = static_cast<size_t>(c->n_total);
  if (!c->d_diag_rec) MD_CUDA(dev_alloc(&c->d_diag_rec, 6 * nt));
  if (c->nseg_used > 1 && c->part_phi_seg < c->nseg_used) {
    cudaFree(c->d_part_phi);
    c->d_part_phi = nullptr;
    MD_CUDA(dev_alloc(&c->d_part_phi, static_cast<size_t>(c->nseg_used) * nt));
    c->part_phi_seg = c->nseg_used;
  }
  MD_CUDA(cudaMemsetAsync(c->d_diag_rec, 0, sizeof(double) * 6 * nt, c->stream));
  long long step = 0;
  MD_CUDA(cudaMemcpyAsync(&step, c->d_step, sizeof(step), cudaMemcpyDeviceToHost, c->stream));
  md::StepArgs a = step_args(c);
  a.diag_rec = c->d_diag_rec;
  a.part_phi = c->d_part_phi;
  MD_CUDA(k.launch_step_pot(a, c->grid, c->stream));
  for (int ci = 0; ci < c->n_clusters; ++ci) {
    md::DiagArgs d;
    d.c = slice_view(c, ci);
    d.x = c->d_x[0];
    d.y = c->d_x[1];
    d.z = c->d_x[2];
    d.ux = c->d_u[0];
    d.uy = c->d_u[1];
    d.uz = c->d_u[2];
    d.qm = c->d_qm;
    d.w = c->d_w;
    d.mass = c->d_mass;
    d.zq = c->d_z;
    d.kind = c->d_kind;
    d.e = nullptr;
    d.phi = nullptr;
    d.step = c->d_step;
    d.part = c->d_part;
    d.rec = c->d_diag_rec;
    MD_CUDA(md::launch_diag(d, c->diag_blocks, c->d_diag, c->stream));
    MD_CUDA(cudaMemcpyAsync(c->h_diag, c->d_diag, sizeof(md::DiagPartial),
                            cudaMemcpyDeviceToHost, c->stream));
    MD_CUDA(cudaStreamSynchronize(c->stream));
    st = check_device_error(c);
    if (st != MD_OK) return st;
    st = fill_diag(*c->h_diag, step, c->cl[ci], &out[ci]);
    if (st == MD_ERR_NONFINITE) worst = st;
  }
  return worst != MD_OK ? fail(worst, "records hold NaN/Inf") : MD_OK;
}

md_status md_step_diag(md_ctx* c, md_diag* out) {
  return md::guarded([&] { return md_step_diag_body(c, out); });
}

static md_status md_get_particles_body(md_ctx* c, int32_t cluster, md_particles* out) {
  if (!c || !out) return fail(MD_ERR_ARG, "NULL argument");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  const long long n = c->cl[cluster].n;
  if (out->n != n) return fail(MD_ERR_ARG, "out->n = %lld, cluster holds %lld", (long long)out->n, n);
  RawView d = raw_view(c->d_raw, n);
  md::DownloadArgs a;
  a.hx = d.x;
  a.hu = d.u;
  a.hz = d.z;
  a.hmass = d.mass;
  a.hw = d.w;
  a.hkind = d.kind;
  a.n = n;
  a.off = c->cl[cluster].off;
  a.x = c->d_x[0];
  a.y = c->d_x[1];
  a.z = c->d_x[2];
  a.ux = c->d_u[0];
  a.uy = c->d_u[1];
  a.uz = c->d_u[2];
  a.w = c->d_w;
  a.mass = c->d_mass;
  a.zq = c->d_z;
  a.kind = c->d_kind;
  MD_CUDA(md::launch_download(a, c->stream));
  // page-locked caller arrays receive their copy directly; the others go
  // through the pinned staging buffer
  RawView h = raw_view(c->h_raw, n);
  struct Part {
    void* user;
    void* stage;
    const void* dev;
    size_t bytes;
    bool direct;
  };
  Part parts[6] = {{out->x, h.x, d.x, sizeof(double) * 3 * n, false},
                   {out->u, h.u, d.u, sizeof(double) * 3 * n, false},
                   {out->z, h.z, d.z, sizeof(int) * n, false},
                   {out->mass, h.mass, d.mass, sizeof(double) * n, false},
                   {out->w, h.w, d.w, sizeof(double) * n, false},
                   {out->kind, h.kind, d.kind, static_cast<size_t>(n), false}};
  for (Part& q : parts) {
    if (!q.user) continue;
    q.direct = is_pinned(q.user);
    MD_CUDA(cudaMemcpyAsync(q.direct ? q.user : q.stage, q.dev, q.bytes, cudaMemcpyDeviceToHost,
                            c->stream));
  }
  MD_CUDA(cudaStreamSynchronize(c->stream));
  for (const Part& q : parts)
    if (q.user && !q.direct) std::memcpy(q.user, q.stage, q.bytes);
  return check_device_error(c);
}

md_status md_get_particles(md_ctx* c, int32_t cluster, md_particles* out) {
  return md::guarded([&] { return md_get_particles_body(c, cluster, out); });
}

static md_status md_set_particles_body(md_ctx* c, int32_t cluster, const md_particles* in) {
  if (!c || !in) return fail(MD_ERR_ARG, "NULL argument");
  if (cluster < 0 || cluster >= c->n_clusters) return fail(MD_ERR_ARG, "bad cluster index");
  if (!c->ion[cluster].rate_model) {
    // the per-record checks run on the staged copy in device memory
    md_status st = check_block(*in, cluster, c->cl[cluster].n);
    if (st != MD_OK) return st;
    return upload_cluster(c, cluster, *in, true);
  }
  md_status st = validate_particles(*in, cluster, c->cl[cluster].n);
  if (st != MD_OK) return st;
  return upload_cluster(c, cluster, *in);
}

md_status md_set_particles(md_ctx* c, int32_t cluster, const md_particles* in) {
  return md::guarded([&] { return md_set_particles_body(c, cluster, in); });
}

int32_t md_tuning_list(md_tuning* list, int32_t cap) {
  int n = 0;
  const md::KernelConfig* cfgs = md::step_configs(&n);
  for (int i = 0; list && i < n && i < cap; ++i) {
    list[i].threads = cfgs[i].threads;
    list[i].r = cfgs[i].r;
    list[i].tile = cfgs[i].tile;
    list[i].ctas_per_sm = 0;
    list[i].jsplit = 0;
    list[i].packed = cfgs[i].packed;
    list[i].min_blocks = cfgs[i].min_blocks;
  }
  return n;
}

static md_status md_set_tuning_body(md_ctx* c, const md_tuning* t) {
  if (!c || !t) return fail(MD_ERR_ARG, "NULL argument");
  int n = 0;
  const md::KernelConfig* cfgs = md::step_configs(&n);
  for (int i = 0; i < n; ++i) {
    if (cfgs[i].threads == t->threads && cfgs[i].r == t->r && cfgs[i].tile == t->tile &&
        cfgs[i].packed == (t->packed != 0) &&
        (t->min_blocks < 0 || cfgs[i].min_blocks == t->min_blocks)) {
      if (t->ctas_per_sm < 0) return fail(MD_ERR_ARG, "ctas_per_sm < 0");
      MD_CUDA(cudaStreamSynchronize(c->stream));
      return configure(c, i, t->ctas_per_sm, t->jsplit);
    }
  }
  return fail(MD_ERR_ARG, "no compiled configuration threads=%d r=%d tile=%d packed=%d",
              t->threads, t->r, t->tile, t->packed);
}

md_status md_set_tuning(md_ctx* c, const md_tuning* t) {
  return md::guarded([&] { return md_set_tuning_body(c, t); });
}

static md_status md_get_tuning_body(md_ctx* c, md_tuning* t) {
  if (!c || !t) return fail(MD_ERR_ARG, "NULL argument");
  int n = 0;
  const md::KernelConfig* cfgs = md::step_configs(&n);
  t->threads = cfgs[c->cfg].threads;
  t->r = cfgs[c->cfg].r;
  t->tile = cfgs[c->cfg].tile;
  t->ctas_per_sm = c->ctas_per_sm;
  t->jsplit = c->jsplit < 0 ? c->jsplit : c->nseg_used;
  t->packed = cfgs[c->cfg].packed;
  t->min_blocks = cfgs[c->cfg].min_blocks;
  return MD_OK;
}

md_status md_get_tuning(md_ctx* c, md_tuning* t) {
  return md::guarded([&] { return md_get_tuning_body(c, t); });
}

static md_status md_plan_shares_body(const int32_t* n_pad, int32_t n_clusters, int32_t per, int32_t tile,
                                     int64_t shares, int32_t* units, int64_t cap, int32_t* first,
                                     int64_t* n_units, int64_t* n_shares) {
  if (!n_pad || !n_units || !n_shares) return fail(MD_ERR_ARG, "NULL argument");
  if (n_clusters < 1 || per < 1 || tile < 1 || shares < 1 || cap < 0)
    return fail(MD_ERR_ARG, "need n_clusters, per, tile, shares >= 1 and cap >= 0");
  if (shares > INT32_MAX) return fail(MD_ERR_ARG, "shares must be below 2^31");
  long long T = 0;
  for (int ci = 0; ci < n_clusters; ++ci) {
    if (n_pad[ci] < 1) return fail(MD_ERR_ARG, "cluster %d: n_pad < 1", ci);
    T += ((static_cast<long long>(n_pad[ci]) + per - 1) / per) *
         ((static_cast<long long>(n_pad[ci]) + tile - 1) / tile);
    if (T > INT32_MAX) return fail(MD_ERR_ARG, "more than 2^31 source tiles in all");
  }
  std::vector<BlockSpan> blks;
  int ib = 0;
  for (int ci = 0; ci < n_clusters; ++ci) {
    const long long nb = (static_cast<long long>(n_pad[ci]) + per - 1) / per;
    const long long tiles = (static_cast<long long>(n_pad[ci]) + tile - 1) / tile;
    for (long long b = 0; b < nb; ++b, ++ib) blks.push_back({ci, static_cast<int>(b), ib, tiles, n_pad[ci]});
  }
  std::vector<md::Unit> us;
  std::vector<int> fs;
  int max_parts = 1;
  const long long G = plan_shares(blks, tile, shares, &us, &fs, &max_parts);
  *n_units = static_cast<int64_t>(us.size());
  *n_shares = G;
  if (!units && !first) return MD_OK;  // a query of the sizes
  if (units && cap < static_cast<int64_t>(us.size()))
    return fail(MD_ERR_ARG, "cap %lld below the %zu units", static_cast<long long>(cap), us.size());
  if (units)
    for (size_t i = 0; i < us.size(); ++i) {
      int32_t* o = units + 6 * i;
      o[0] = us[i].cluster;
      o[1] = us[i].block;
      o[2] = us[i].seg;
      o[3] = us[i].nparts;
      o[4] = us[i].j0;
      o[5] = us[i].jn;
    }
  if (first)
    for (size_t i = 0; i < fs.size(); ++i) first[i] = fs[i];
  return MD_OK;
}

md_status md_plan_shares(const int32_t* n_pad, int32_t n_clusters, int32_t per, int32_t tile,
                         int64_t shares, int32_t* units, int64_t cap, int32_t* first,
                         int64_t* n_units, int64_t* n_shares) {
  return md::guarded([&] { return md_plan_shares_body(n_pad, n_clusters, per, tile, shares, units, cap, first, n_units, n_shares); });
}

static md_status md_autotune_body(md_ctx* c, int32_t steps, double* times_ms, int32_t cap) {
  if (!c) return fail(MD_ERR_ARG, "ctx is NULL");
  if (steps < 1) return fail(MD_ERR_ARG, "steps < 1");
  const size_t N = static_cast<size_t>(c->n_total);
  const size_t G = static_cast<size_t>((c->n_total + md::kLiveGroup - 1) / md::kLiveGroup);
  // every mutable device array of the state (ionization changes charges,
  // kinds, weights and flags as well): backed up, restored after each trial
  struct Buf {
    void* dev;
    size_t bytes;
    void* copy;
  };
  std::vector<Buf> bufs = {{c->d_posq[0], N * sizeof(float4), nullptr},
                           {c->d_posq[1], N * sizeof(float4), nullptr},
                           {c->d_qm, N * sizeof(float), nullptr},
                           {c->d_w, N * sizeof(double), nullptr},
                           {c->d_mass, N * sizeof(double), nullptr},
                           {c->d_z, N * sizeof(int), nullptr},
                           {c->d_kind, N, nullptr}};
  for (int k = 0; k < 3; ++k) {
    bufs.push_back({c->d_x[k], N * sizeof(double), nullptr});
    bufs.push_back({c->d_u[k], N * sizeof(double), nullptr});
  }
  if (c->d_src_live) {
    bufs.push_back({c->d_src_live, G, nullptr});
    bufs.push_back({c->d_tgt_live, G, nullptr});
  }
  if (c->d_vel) bufs.push_back({c->d_vel, N * sizeof(float4), nullptr});
  if (c->d_ion_next)
    bufs.push_back({c->d_ion_next, sizeof(long long) * c->n_clusters, nullptr});
  if (c->d_det_hist) {
    bufs.push_back({c->d_det_hist, sizeof(unsigned long long) * c->n_clusters * 5 *
                                       (kDetMaxBins + 1), nullptr});
    bufs.push_back({c->d_det_crossed, N, nullptr});
  }
  auto release = [&]() {
    for (auto& b : bufs) cudaFree(b.copy);
  };
  for (auto& b : bufs) {
    if (cudaMalloc(&b.copy, b.bytes) != cudaSuccess) {
      release();
      return fail(MD_ERR_OOM, "autotune backup allocation failed");
    }
  }
  cudaStream_t s = c->stream;
  long long step0 = 0;
  for (auto& b : bufs) cudaMemcpyAsync(b.copy, b.dev, b.bytes, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(&step0, c->d_step, sizeof(step0), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  const int cfg0 = c->cfg, cps0 = c->ctas_per_sm, js0 = c->jsplit;
  int n = 0;
  const md::KernelConfig* cfgs = md::step_configs(&n);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  int best_cfg = cfg0, best_js = 0;
  md_status st = MD_OK;
  std::vector<double> by_cfg(static_cast<size_t>(n), -1.0);
  // one trial: configuration i with source split js, timed over `steps`
  // steps from the saved state (restored afterwards)
  auto trial = [&](int i, int js) {
    st = configure(c, i, 0, js);
    if (st != MD_OK) return;
    st = launch_steps_direct(c, 1);  // warm-up
    if (st != MD_OK) return;
    cudaEventRecord(e0, s);
    st = launch_steps_direct(c, steps);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(MD_ERR_CUDA, "autotune timing");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / steps;
    if (by_cfg[i] < 0.0 || per < by_cfg[i]) by_cfg[i] = per;
    if (per < best) {
      best = per;
      best_cfg = i;
      best_js = js;
    }
    if (st == MD_OK) st = check_device_error(c);
    for (auto& b : bufs) cudaMemcpyAsync(b.dev, b.copy, b.bytes, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->d_step, &step0, sizeof(step0), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  };
  // every configuration with its segments chosen for balance, then the two
  // fastest with equal shares (each count of kAutoShares per resident CTA),
  // which fill the last round of a large step but add pieces that cross
  // i-blocks
  for (int i = 0; i < n && st == MD_OK; ++i) {
    int bps = 0;
    if (c->any_mi && !cfgs[i].launch_step_mi) continue;  // no minimum-image kernel
    if (blocks_per_sm_of(c, cfgs[i], &bps) != cudaSuccess || bps < 1) continue;  // does not fit
    trial(i, 0);
  }
  if (st == MD_OK && !any_ionizing(c)) {
    std::vector<int> order;
    for (int i = 0; i < n; ++i)
      if (by_cfg[i] >= 0.0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return by_cfg[x] < by_cfg[y]; });
    for (size_t k = 0; k < order.size() && k < 2 && st == MD_OK; ++k)
      for (int sh : kAutoShares)
        if (st == MD_OK) trial(order[k], -sh);
  }
  if (times_ms)
    for (int i = 0; i < n && i < cap; ++i) times_ms[i] = by_cfg[i];
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (st != MD_OK) {
    configure(c, cfg0, cps0, js0);
    return st;
  }
  return configure(c, best_cfg, 0, best_js);
}

md_status md_autotune(md_ctx* c, int32_t steps, double* times_ms, int32_t cap) {
  return md::guarded([&] { return md_autotune_body(c, steps, times_ms, cap); });
}

static md_status md_coulomb_field_fp64_device_body(const double* xs, const double* qs, int64_t ns,
                                                   const double* xt, const int64_t* self_idx, int64_t nt,
                                                   double eps, double kc, double* e, double* phi,
                                                   void* stream) {
  if (ns < 0 || nt < 0) return fail(MD_ERR_ARG, "negative size");
  if (nt == 0) return MD_OK;
  if (!xs || !qs || !xt || !e) return fail(MD_ERR_ARG, "NULL pointer");
  if (!(eps >= 0.0) || !(kc > 0.0)) return fail(MD_ERR_ARG, "eps must be >= 0 and kc > 0");
  MD_CUDA(md::launch_field_fp64(xs, qs, ns, xt, reinterpret_cast<const long long*>(self_idx), nt,
                                eps, kc, e, phi, static_cast<cudaStream_t>(stream)));
  return MD_OK;
}

md_status md_coulomb_field_fp64_device(const double* xs, const double* qs, int64_t ns,
                                       const double* xt, const int64_t* self_idx, int64_t nt,
                                       double eps, double kc, double* e, double* phi,
                                       void* stream) {
  return md::guarded([&] { return md_coulomb_field_fp64_device_body(xs, qs, ns, xt, self_idx, nt, eps, kc, e, phi, stream); });
}

static md_status md_coulomb_field_device_body(const void* src, int64_t ns, const void* tgt, int64_t nt,
                                              float eps2, int64_t self_offset, double* e, double* phi,
                                              void* stream) {
  if (ns < 0 || nt < 0) return fail(MD_ERR_ARG, "negative size");
  if (nt == 0) return MD_OK;
  if (!src || !tgt || !e) return fail(MD_ERR_ARG, "NULL pointer");
  if ((reinterpret_cast<uintptr_t>(src) & 15) || (reinterpret_cast<uintptr_t>(tgt) & 15))
    return fail(MD_ERR_ARG, "src and tgt must be 16-byte aligned");
  if (!(eps2 > 0.0f)) return fail(MD_ERR_ARG, "eps2 must be > 0");
  // the sticky error word of the stateless field calls on this device, read
  // and cleared by md_field_device_status
  int dev = 0;
  MD_CUDA(cudaGetDevice(&dev));
  int* d_err = nullptr;
  {
    const md_status es = md::field_error_word(&d_err);
    if (es != MD_OK) return es;
  }
  md::FieldArgs a;
  a.src = static_cast<const float4*>(src);
  a.ns = ns;
  a.tgt = static_cast<const float4*>(tgt);
  a.nt = nt;
  a.eps2 = eps2;
  a.self_offset = self_offset;
  a.e = e;
  a.phi = phi;
  a.err = d_err;
  a.src_live = nullptr;
  a.tgt_live = nullptr;
  a.gbase = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // split the sources until about 4 waves of CTAs run (up to 64 segments of
  // at least 4 tiles, partials of at most 256 MB); the partials live in
  // stream-ordered memory, so calls on different streams do not share them
  int bps = 1, sms = 1;
  MD_CUDA(md::field_blocks_per_sm(&bps));
  MD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long per = md::field_targets_per_cta();
  const long long nt_ = static_cast<long long>(nt), ns_ = static_cast<long long>(ns);
  const long long blocks = (nt_ + per - 1) / per;
  const long long want = (4LL * std::max(1, bps) * sms + blocks - 1) / blocks;
  const long long by_mem = (256LL << 20) / (32LL * nt_);
  const long long nseg = std::max(1LL, std::min({want, 64LL, ns_ / 2048, by_mem}));
  void* part = nullptr;
  if (nseg > 1) {
    MD_CUDA(cudaMallocAsync(&part, static_cast<size_t>(32 * nseg * nt_), st));
    a.nseg = static_cast<int>(nseg);
    a.seg_len = (ns_ + nseg - 1) / nseg;
    a.part = static_cast<double*>(part);
  }
  const cudaError_t le = md::launch_field(a, phi != nullptr, st);
  if (part) MD_CUDA(cudaFreeAsync(part, st));
  MD_CUDA(le);
  return MD_OK;
}

md_status md_coulomb_field_device(const void* src, int64_t ns, const void* tgt, int64_t nt,
                                  float eps2, int64_t self_offset, double* e, double* phi,
                                  void* stream) {
  return md::guarded([&] { return md_coulomb_field_device_body(src, ns, tgt, nt, eps2, self_offset, e, phi, stream); });
}

static md_status md_measure_fp32_peak_body(double* ffma_per_s, double* packed_fma_per_s, void* stream) {
  if (!ffma_per_s) return fail(MD_ERR_ARG, "NULL argument");
  int dev = 0, sms = 0;
  MD_CUDA(cudaGetDevice(&dev));
  MD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* sink = nullptr;
  MD_CUDA(cudaMalloc(reinterpret_cast<void**>(&sink), sizeof(float) * 8 * sms));
  const int blocks = 8 * sms, iters = 20000;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double rate[2] = {0.0, 0.0};
  cudaError_t e = cudaSuccess;
  for (int packed = 0; packed < 2 && e == cudaSuccess; ++packed) {
    e = md::launch_ffma_probe(blocks, iters / 10, packed != 0, sink, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = md::launch_ffma_probe(blocks, iters, packed != 0, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    // lane FMAs: 256 threads x iters x 16 x 8 chains (x 2 lanes when packed)
    const double fma = static_cast<double>(blocks) * 256.0 * iters * 128.0 * (packed ? 2.0 : 1.0);
    rate[packed] = fma / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "FP32 peak probe");
  *ffma_per_s = rate[0];
  if (packed_fma_per_s) *packed_fma_per_s = rate[1];
  return MD_OK;
}

md_status md_measure_fp32_peak(double* ffma_per_s, double* packed_fma_per_s, void* stream) {
  return md::guarded([&] { return md_measure_fp32_peak_body(ffma_per_s, packed_fma_per_s, stream); });
}

}  // extern "C"
