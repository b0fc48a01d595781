// md_types.cuh -- plain data shared by the kernels and the host runtime.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace md {

constexpr int kPad = 16;                          // records per cluster padded to a multiple of this
constexpr long long kWaitBudget = 4000000000LL;   // clock64 cycles (about 2 s)
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;   // a bounds check of the checked build failed
constexpr int kHistBins = 16;
constexpr int kLiveGroup = 64;  // records per liveness flag

struct ClusterDev {
  long long off;   // first record of the cluster
  int n;           // real records
  int n_pad;       // records incl. zero-charge padding (multiple of kPad)
  int nseg;        // sources split into nseg segments (work units) per i-block
  int seg_len;     // sources per segment (last one shorter); with equal shares
                   // the units carry their own source pieces and nseg is 1
  double a0, tau, t0, dt, box, t_switch;
  float eps2;
  int pol, env, boundary;
  // ion energy detectors on the sphere |x - det_c| = sqrt(det_r2) (off: det_nbins = 0)
  int det_nbins;
  double det_r2, det_cos, det_emax, det_c[3];
  long long det_off;  // first histogram entry of the cluster (5 x (det_nbins + 1) entries)
};

// Segment length that splits the live records [0, live) of a cluster of
// n_pad records into nseg source segments of the step (a multiple of kPad).
// It is at most the split of all n_pad records, so every segment starts
// inside the cluster; the step's segments cover [0, live) whole.
__host__ __device__ inline int live_seg_len(int n_pad, int nseg, long long live) {
  nseg = nseg < 1 ? 1 : nseg;
  live = live < 0 ? 0 : (live > n_pad ? n_pad : live);
  long long len = (live + nseg - 1) / nseg;
  len = (len + kPad - 1) / kPad * kPad;
  return static_cast<int>(len < kPad ? kPad : len);
}

constexpr int kMaxZ = 16;
constexpr int kIonScratch = 11;   // doubles per ion and source segment
constexpr int kIonMaxSeg = 32;    // source segments of the ionization field pass

// Ionization parameters of one cluster (Sec. II, ionization paragraph).
struct IonDev {
  int rate_model;     // 0 off, 1 ADK + Lotz, 2 MLP surrogate (1 outside its range)
  int ionize_every;   // pass before every k-th step (0: explicit calls only)
  int zmax;
  int n_ions;         // records [off, off + n_ions) can ionize
  long long slot_base;  // cluster-relative first electron slot (filled densely)
  unsigned long long seed;
  double r_loc, r_create;
  double kc;          // K_C of the cluster: Q = kc w z
  double k_si;        // laser wave number, 1/m
  double omega;       // laser angular frequency, rad/s
  double ip_ev[kMaxZ];
  double q_outer[kMaxZ];
  double dom[6];      // surrogate domain: |E| min/max, n_e min/max, T_e min/max
};

// One unit of the step kernel: the field at one i-block of targets from one
// piece of its cluster's sources.  The pieces of an i-block publish partial
// fields that the last of them adds up in piece order.
struct Unit {
  int cluster;
  int block;   // i-block within the cluster
  int seg;     // piece of the i-block's sources
  int ib;      // i-block index over all clusters (completion counter)
  int j0;      // first source record of the piece, and
  int jn;      // its length; jn < 0: piece seg of the cluster's nseg segments
               // of seg_len records (a split the device may reset, R16)
  int nparts;  // pieces of this i-block (jn >= 0)
  int pad_;
};

struct StepArgs {
  const ClusterDev* cl;
  const Unit* units;
  // shares of the work handed out by the ticket: share k runs the units
  // [share_first[k], share_first[k + 1]) in order
  const int* share_first;
  int n_shares;
  float4* posq0;
  float4* posq1;
  double* x;
  double* y;
  double* z;
  double* ux;
  double* uy;
  double* uz;
  const float* qm;
  long long* step;
  unsigned* ticket;
  unsigned* done;
  int* err;
  // split sources: partial fields [seg][n_total][3] and per-i-block counters
  double* part;
  unsigned* iblk_cnt;
  long long n_total;
  // liveness per group of kLiveGroup records (nullptr: everything live):
  // src_live = some record carries charge, tgt_live = some record is active
  const unsigned char* src_live;
  const unsigned char* tgt_live;
  // FP32 copy (ux, uy, uz, w) of every record's u and weight, read by the
  // ionization pass for the local electron moments (nullptr: not kept)
  float4* vel;
  // ion energy detectors (nullptr: none configured)
  unsigned long long* det_hist;
  unsigned char* det_crossed;
  const double* mass;
  // diagnostic steps only (the POT step kernel): per record (status, ke, pe,
  // px, py, pz) at t_n, [n_total][6], and the potential partials of split
  // sources, [nseg][n_total]
  double* diag_rec;
  double* part_phi;
  const int* zq;
  const unsigned char* kind;
  const double* w;
  // per cluster: minimum-image forces while periodic (nullptr: no cluster)
  const unsigned char* min_image;
};

// Cell list of the electrons near the ions, for the local moments of the
// ionization pass (clusters without minimum-image forces): cells of side
// 1.01 r_loc, hashed into kCellBuckets buckets, the electrons of each bucket
// listed contiguously as (position record, velocity record) pairs, and the
// ions listed by bucket too.
constexpr int kCellBuckets = 1 << 18;
struct CellBuf {
  int* count;    // [kCellBuckets] electrons per bucket
  int* start;    // [kCellBuckets + 1] first listed electron of each bucket
  int* fill;     // [kCellBuckets] fill counters of the listing
  float4* rec;   // [2 capacity] the listed electrons' position and velocity records
  long long capacity;
  // the ions listed by bucket, so that neighbouring threads of the moment
  // kernel take ions of one cell and read the same electron lists
  int* ion_count;  // [kCellBuckets]
  int* ion_start;  // [kCellBuckets + 1]
  int* ion_fill;   // [kCellBuckets]
  int* ion_list;   // [n_ions capacity] ion records in bucket order
  int* scan_tmp;   // [kCellBuckets / 1024] block totals of the bucket scans
};

// Arguments of the ionization kernels of one cluster.
struct IonArgs {
  ClusterDev c;
  IonDev ion;
  float4* posq0;
  float4* posq1;
  double* x;
  double* y;
  double* z;
  double* ux;
  double* uy;
  double* uz;
  float* qm;
  double* w;
  double* mass;
  int* zq;
  unsigned char* kind;
  const long long* step;
  int* err;
  int force;          // 1: run regardless of ionize_every
  double* scratch;    // [nseg][n_ions][kIonScratch]: ex, ey, ez, sw, sw du_x, sw du_y,
                      // sw du_z, sw du^2, u_ref (3) of each source segment (du = u -
                      // u_ref, u_ref = the segment's first local electron's u)
  int nseg;           // source segments of the field pass (equal shares of the live records)
  int* blk_fired;     // [ceil(n_ions / 256)] fired ions per block of the decision
  long long* pass_slot;  // first free slot at the start of the pass
  double* out;        // [n_ions][4]: |E|, ne (cm^-3), Te (eV), P
  double* nu;         // [n_ions]: rate from the surrogate, or -1 (use the plain rate)
  unsigned char* fired;  // [n_ions]
  const float* mlp;   // surrogate weights (rate_model 2) or nullptr
  unsigned char* src_live;  // liveness flags (set when a record becomes charged / active)
  unsigned char* tgt_live;
  float4* vel;        // FP32 (ux, uy, uz, w) per record
  long long* next_slot;  // cluster-relative record of the next free electron slot
  // this cluster's descriptor on the device: the pass that moves next_slot
  // also resets its seg_len to the split of the live records (live_seg_len)
  ClusterDev* cl_dev;
  // clusters with a pass before every step (nullptr otherwise): the Coulomb
  // field at each ion after the pass's charge changes, [n_ions][3], which the
  // step uses for the ions instead of summing their field again; and the
  // pass's charge changes as two source streams in slot order, [2 n_ions]:
  // fix_src[k] = (x, y, z, +K_C w) of the k-th fired ion (its extra charge),
  // fix_src[n_ions + k] = its freed electron's j-stream record
  double* e_ion;
  float4* fix_src;
  int fix_nseg;       // source segments of the charge-change field (k_ion_fix)
  // local moments from a cell list (cells.count non-null) instead of beside
  // the field sum
  CellBuf cells;
  // 1: minimum-image distances while the boundary is periodic (field and
  // local moments of the pass, charge-change correction)
  int min_image;
};

struct FieldArgs {
  const float4* src;
  long long ns;
  const float4* tgt;
  long long nt;
  float eps2;
  long long self_offset;  // target i is source i + self_offset, or -1
  double* e;              // [nt][3]
  double* phi;            // [nt] or nullptr
  int* err;
  // liveness flags of the context (nullptr: everything live); source record j
  // and target record i are global records gbase + j and gbase + i
  const unsigned char* src_live;
  const unsigned char* tgt_live;
  long long gbase;
  // sources split into nseg segments of seg_len (nseg > 1): CTA (x, y) sums
  // segment y into part[y][nt][4] = (ex, ey, ez, phi), and a second kernel
  // adds the segments in order
  int nseg = 1;
  long long seg_len = 0;
  double* part = nullptr;
  // > 0: minimum-image displacements in the periodic cube of this side
  float box = 0.0f;
};

struct DiagPartial {
  double v[8];  // ke, ke_ions, ke_electrons, pe, px, py, pz, unused
  long long cnt[2];  // n_active, n_nonfinite
  long long hist[kHistBins];
  double histw[kHistBins];
};
constexpr int kDiagVals = 8 + 2 + 2 * kHistBins;

struct DiagArgs {
  ClusterDev c;
  const double* x;
  const double* y;
  const double* z;
  const double* ux;
  const double* uy;
  const double* uz;
  const float* qm;
  const double* w;
  const double* mass;
  const int* zq;
  const unsigned char* kind;
  const double* e;    // Coulomb field [n_pad][3] of this cluster
  const double* phi;  // potential [n_pad]
  const long long* step;
  DiagPartial* part;  // [gridDim.x]
  // per-record diagnostics of a diagnostic step ([n_total][6], status, ke,
  // pe, px, py, pz), used instead of e / phi and the kick; or nullptr
  const double* rec = nullptr;
};

struct UploadArgs {
  const double* hx;
  const double* hu;
  const int* hz;
  const double* hmass;
  const double* hw;
  const unsigned char* hkind;
  long long n;
  long long off;
  double kc;
  float4* posq0;
  float4* posq1;
  double* x;
  double* y;
  double* z;
  double* ux;
  double* uy;
  double* uz;
  float* qm;
  double* w;
  double* mass;
  int* zq;
  unsigned char* kind;
  const long long* step;
  float4* vel;        // FP32 (ux, uy, uz, w) or nullptr
  // index of the first record k_validate rejected (kNoBadRecord: none), or
  // nullptr: the records were checked on the host.  A rejected block is not
  // applied.
  unsigned long long* first_bad;
};

constexpr unsigned long long kNoBadRecord = ~0ull;

// Seeded generation of one cluster's records into the host-layout staging
// buffer (x[n][3], u[n][3], mass, w, z, kind), which k_upload then scatters.
struct GenerateArgs {
  double r0;
  double c[3];          // sphere centre
  double ion_mass;
  double weight;
  double sig_i, sig_e;  // per-component spread of u of ions / electrons (0: at rest)
  long long n_ions, n_electrons, n;  // n = n_ions + n_electrons + slots
  int ion_charge;
  unsigned long long seed;
  double* x;
  double* u;
  double* mass;
  double* w;
  int* z;
  unsigned char* kind;
};

struct DownloadArgs {
  double* hx;
  double* hu;
  int* hz;
  double* hmass;
  double* hw;
  unsigned char* hkind;
  long long n;
  long long off;
  const double* x;
  const double* y;
  const double* z;
  const double* ux;
  const double* uy;
  const double* uz;
  const double* w;
  const double* mass;
  const int* zq;
  const unsigned char* kind;
};

}  // namespace md
