// FP64 instantiations of the sweep kernel.
#define HZ_SWEEP_REAL double
#define HZ_SWEEP_LAUNCHER launch_sweep_f64
#include "hz_sweep_impl.cuh"
