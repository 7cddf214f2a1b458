// Launchers of the device kernels (private to the library).
#pragma once
#include <cuda_runtime.h>

#include "view.h"

namespace spider {

// message returned by spider_last_error(NULL)
void set_static_error(const char* msg);

// travel times (k_tt.cu, k_mlp_tc.cu)
bool tt_supported_width(int H);
size_t tt_scratch_floats(const NetView& net, int num_sms);
// ctas_per_sm (1 or 2) shapes the FP32 MLP grid; scratch holds 2 x num_sms slots
cudaError_t launch_tt(const NetView& net, const PairSource& src, TTOut out, int num_sms, float* scratch,
                      cudaStream_t st, int ctas_per_sm);
cudaError_t launch_mlp_tc(const NetView& net, const PairSource& src, TTOut out, int num_sms,
                          float* scratch, cudaStream_t st);
bool mlp_tc_supported(int H, int precision);
// builds the tensor-core operand images (the first layer's split BF16 image,
// then the hidden layers) on the device
cudaError_t mlp_tc_prepare(const float* W1_host, const float* const Wn_host[3], const float* w5_host, int H,
                           int precision, void** image, float** scales, cudaStream_t st);

// step (k_step.cu)
cudaError_t configure_step_kernels(const StepView& v);
int pcg_grid(const StepView& v, int num_sms);
cudaError_t launch_select(const StepView& v, int64_t n_b, cudaStream_t st, int bthreads = 256);
// bthreads: threads per CTA of the per-block kernels k_resid and k_final (a
// multiple of 32 up to 1024; results do not depend on it except the rounding
// order of the FP64 r.q sums)
cudaError_t launch_resid(const StepView& v, int64_t n_b, int gu, cudaStream_t st, const cudaEvent_t* ev,
                         int bthreads = 256);
cudaError_t launch_pcg(const StepView& v, int64_t n_b, int max_it, float tol, int grid, int warp_mult,
                       int cta_mult, cudaStream_t st);
cudaError_t launch_finish(const StepView& v, int64_t n_b, int gu, bool logpost, cudaStream_t st,
                          const cudaEvent_t* ev, int bthreads = 256);
// theta_0 + state (or a stored sample) in FP64, caller order (M x 4)
cudaError_t launch_state_out(const StepView& v, const float4* src, double* out, int grid, cudaStream_t st);
// the last gradient (FP32), caller order (M x 4)
cudaError_t launch_grad_out(const StepView& v, float4* out, int grid, cudaStream_t st);
cudaError_t launch_diag(const StepView& v, const float4* g, const float4* G, double* norms, double* part,
                        int grid, cudaStream_t st);
// whitening through the precomputed piece inverses (k_whiten.cu)
int piece_max_nodes();
int64_t whiten_unit_scratch_floats();   // global scratch per CTA of the unit solver
cudaError_t configure_whiten_kernels();
int whiten_units_grids(int num_sms, int grids[3]);
int piece_cc_grid(int num_sms);
int whiten_clean_grid(int num_sms);
// branch streams on which independent kernels of one stage run side by side:
// `fork` is recorded on the launching stream and waited on by each branch,
// join[i] is recorded on branch i and waited on by the launching stream
struct Branches {
  cudaStream_t s[4];
  cudaEvent_t fork;
  cudaEvent_t join[4];
};
// the units of a step, data-parallel (k_units.cu); br (nullable): the size
// classes of the small inverses run concurrently on its streams
cudaError_t launch_units(const StepView& v, float tol, int num_sms, cudaStream_t st, cudaEvent_t mid = nullptr,
                         const Branches* br = nullptr);
cudaError_t configure_units_kernels();
// ev (nullable): five events recorded on st after the piece labelling, the
// units' set-up, their refinement rounds, the CTA unit passes and the join
// with the clean-piece solver (timed evaluations only)
cudaError_t launch_whiten_fast(const StepView& v, int64_t n_b, float tol, int cc_grid, const int grids[4],
                               int clean_grid, cudaStream_t st, cudaStream_t side, cudaEvent_t fork,
                               cudaEvent_t join, const cudaEvent_t* ev = nullptr, int clean_share = 4,
                               const Branches* br = nullptr);
// stage-1 outlier mask (k_outlier.cu)
size_t outlier_scratch_bytes(int n_sub);
cudaError_t launch_outlier(const StepView& v, int n_sub, float kmad, void* scratch, uint8_t* keep,
                           int num_sms, cudaStream_t st, float* med_host, float* mad_host, int64_t* n_kept);
cudaError_t launch_linfilter(const StepView& v, int64_t n_b, float max_rel, uint8_t* keep,
                             unsigned long long* kept, cudaStream_t st);
// posterior summaries (k_uq.cu)
int uq_max_samples();
cudaError_t launch_uq(const StepView& v, int64_t first, int n, const double* truth_off, double lo_pct,
                      double hi_pct, double* med, double* half, double* calib, double* ess, cudaStream_t st);
cudaError_t launch_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                int64_t n, uint32_t* out, cudaStream_t st);

}  // namespace spider
