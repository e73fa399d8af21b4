// FP32 instantiations of the sweep kernel (subdomain WaveHoltz loop in single
// precision; the outer iteration stays FP64).
#define HZ_SWEEP_REAL float
#define HZ_SWEEP_LAUNCHER launch_sweep_f32
#include "hz_sweep_impl.cuh"
