// md_internal.h -- interface between the kernel instantiations (md_kernels.cu)
// and the host runtime (md_runtime.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <new>

#include "md.h"
#include "md_types.cuh"

namespace md {

// One compiled configuration of the fused step kernel.
struct KernelConfig {
  int threads;
  int r;
  int tile;
  int stages;
  int packed;      // pair arithmetic in packed f32x2
  int min_blocks;  // launch bound: CTAs per SM the register budget is sized for
  cudaError_t (*launch_step)(const StepArgs& a, int grid, cudaStream_t s);
  cudaError_t (*max_blocks_per_sm)(int* out);
  // the same configuration compiled with the ion energy detectors in the
  // epilogue (used while any cluster of the context has detectors)
  cudaError_t (*launch_step_det)(const StepArgs& a, int grid, cudaStream_t s);
  cudaError_t (*max_blocks_per_sm_det)(int* out);
  // the diagnostic step (potential and per-record diagnostics at t_n), or
  // nullptr (packed configurations)
  cudaError_t (*launch_step_pot)(const StepArgs& a, int grid, cudaStream_t s);
  cudaError_t (*max_blocks_per_sm_pot)(int* out);
  // minimum-image forces for periodic clusters that ask for them, or nullptr
  // (packed configurations)
  cudaError_t (*launch_step_mi)(const StepArgs& a, int grid, cudaStream_t s);
  cudaError_t (*max_blocks_per_sm_mi)(int* out);
  // the same with the detector epilogue
  cudaError_t (*launch_step_mi_det)(const StepArgs& a, int grid, cudaStream_t s);
  cudaError_t (*max_blocks_per_sm_mi_det)(int* out);
};

const KernelConfig* step_configs(int* count);

// Field (and potential) at nt targets from ns sources (FP32/Kahan direct sum),
// with the sources split as a.nseg / a.seg_len / a.part say.
cudaError_t launch_field(const FieldArgs& a, bool potential, cudaStream_t s);
int field_targets_per_cta();
cudaError_t field_blocks_per_sm(int* out);

// Diagnostics: per-block partials then a deterministic final sum.
constexpr int kDiagThreads = 256;
cudaError_t launch_diag(const DiagArgs& a, int blocks, DiagPartial* out, cudaStream_t s);

// FP32 peak probe: blocks x 256 threads x iters x 128 FFMA each (scalar
// fma.rn.f32, or packed fma.rn.f32x2 doing two lanes per instruction).
cudaError_t launch_ffma_probe(int blocks, int iters, bool packed, float* sink, cudaStream_t s);

// Staged records -> state.  With a.first_bad set, k_validate checks every
// record first and a rejected block is not applied.
cudaError_t launch_upload(const UploadArgs& a, cudaStream_t s);

// Seeded records of one cluster into the host-layout staging buffer.
cudaError_t launch_generate(const GenerateArgs& g, cudaStream_t s);

// Count of the records [off, off + n) that are not INACTIVE, into *out.
cudaError_t launch_count_active(const unsigned char* kind, long long off, long long n,
                                unsigned long long* out, cudaStream_t s);

// Launches one CTA whose mbarrier wait can never complete (bounded by budget).
cudaError_t launch_wait_selftest(long long budget, int* err, cudaStream_t s);

// Ionization pass of one cluster: field + local moments, then the decision.
cudaError_t launch_ion_pass(const IonArgs& a, cudaStream_t s);

// Push of the first n_push ion records of cluster ci with the field the
// ionization pass left in e_ion (clusters with a pass before every step; the
// step kernel's units skip their i-blocks).  Launched after the pass and
// before the step kernel.
cudaError_t launch_ion_push(const StepArgs& a, int ci, const double* e_ion, long long n_push,
                            bool det, cudaStream_t s);

// Shape of the field + moments kernel: ion targets per CTA and resident CTAs
// per SM (for the choice of the source split).
int ion_field_targets_per_cta();
cudaError_t ion_field_blocks_per_sm(int* out);
// Shape of the charge-change field kernel (k_ion_fix): ion targets per CTA and
// resident CTAs per SM.
int ion_fix_targets_per_cta();
cudaError_t ion_fix_blocks_per_sm(int* out);
// Shape of the field-only pass kernel (clusters whose moments come from the
// cell list).
int ion_sum_targets_per_cta();
cudaError_t ion_sum_blocks_per_sm(int* out);

// Liveness flags of all records (contexts with ionization).
cudaError_t launch_live_init(const float4* posq0, const float4* posq1, const unsigned char* kind,
                             const long long* step, long long n_total, unsigned char* src_live,
                             unsigned char* tgt_live, cudaStream_t s);

// Surrogate rates of the ions inside its domain (rate_model 2).
cudaError_t launch_ion_mlp(const IonArgs& a, cudaStream_t s);

// Device address of the current device's error word of the stateless field
// calls (a file-scope device array, looked up once per device).
md_status field_error_word(int** out);

// Records the thread-local message returned by md_last_error() and returns
// the status (implemented in md_runtime.cu).
md_status report_error(md_status status, const char* msg);

// Runs an entry point's body: the C ABI returns a status and lets no C++
// exception out (a host allocation that fails becomes MD_ERR_OOM).
template <class F>
md_status guarded(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return report_error(MD_ERR_OOM, "host memory allocation failed");
  } catch (...) {
    return report_error(MD_ERR_STATE, "unexpected host exception");
  }
}
md_status report_cuda_error(cudaError_t e, const char* what);
cudaError_t launch_download(const DownloadArgs& a, cudaStream_t s);

// FP64 reference direct sum (see md_coulomb_field_fp64_device).
cudaError_t launch_field_fp64(const double* xs, const double* qs, long long ns, const double* xt,
                              const long long* self_idx, long long nt, double eps, double kc,
                              double* e, double* phi, cudaStream_t s);

// Energy histogram [det_nbins + 1] of the cluster's ions not recorded by the
// detectors (added to `hist`).
cudaError_t launch_iedf_inside(const ClusterDev& c, const double* ux, const double* uy,
                               const double* uz, const double* mass, const int* zq,
                               const unsigned char* kind, const unsigned char* crossed,
                               unsigned long long* hist, cudaStream_t s);

}  // namespace md
