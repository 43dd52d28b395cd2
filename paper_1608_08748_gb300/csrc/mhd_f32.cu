// mhd_f32.cu -- FP32-bulk instances of the runtime launchers (reconstruction, fluxes and updates
// in float; the CFL reduction, chemistry and diagnostics sums stay FP64 inside the kernels).  This
// translation unit is compiled with FMA contraction on: the FP32 path is compared with the FP64
// oracle against a tolerance, not bit for bit.
#define MHD_RT_F32_TU
#include "mhd_runtime.cuh"

namespace mhd_rt {
// index-check flags of the FP32-bulk kernels (MHD_CHECK builds)
unsigned check_flags_f32(bool clear) { return check_flags_of_this_unit(clear); }

template cudaError_t prepare_kernels<float>();
template void launch_euler_stage<float>(Exec<float>&, cudaStream_t);
template void launch_lag_stage<float>(Exec<float>&, cudaStream_t, bool);
template void launch_step<float>(Exec<float>&, cudaStream_t);
template void launch_post<float>(Exec<float>&, cudaStream_t, int, int, int);
template cudaError_t launch_cfl<float>(Exec<float>&, cudaStream_t);
template cudaError_t launch_set_params<float>(Exec<float>&, cudaStream_t, double, double, int, double);
template void launch_small<float>(Exec<float>&, cudaStream_t, int, double, double, int, double);
template cudaError_t load_state<float, double>(mhd_sim*, Box<float>&, const double* const*);
template cudaError_t load_state<float, float>(mhd_sim*, Box<float>&, const float* const*);
template cudaError_t store_state<float, double>(mhd_sim*, Box<float>&, double* const*);
template cudaError_t store_state<float, float>(mhd_sim*, Box<float>&, float* const*);
template cudaError_t set_faces<float>(mhd_sim*, Box<float>&, const double* const*);
template cudaError_t store_full<float>(mhd_sim*, Box<float>&, double* const*);
template cudaError_t load_full<float>(mhd_sim*, Box<float>&, const double* const*);
template cudaError_t diag_partial<float>(mhd_sim*, Box<float>&);
template cudaError_t store_ions<float>(mhd_sim*, Box<float>&, double*);
template cudaError_t load_ions<float>(mhd_sim*, Box<float>&, const double*);
}  // namespace mhd_rt
