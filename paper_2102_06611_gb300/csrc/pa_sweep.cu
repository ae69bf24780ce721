// pa_sweep.cu -- the sweep kernels of a single run with the Metropolis update: step 1
// (simple-sampling initialisation) and step 3 (theta checkerboard sweeps), each fused with
// the measurement (the kernel template is in pa_sweep.cuh; heatbath instantiations are in
// pa_sweep_hb.cu; the persistent sweep kernels of batches are in pa_batch_sweep.cu).
#include "pa_sweep.cuh"

namespace pa {

bool sweep_has_template(int L)
{
    switch (L) {
        case 4: case 8: case 12: case 16: case 20: case 24: case 32: case 40: case 48: case 64: case 80: case 96:
        case 128:
            return true;
        default: return false;
    }
}

cudaError_t launch_sweep(int L, bool init, const SweepArgs &a, int num_sms, cudaStream_t s)
{
    if (!sweep_has_template(L)) return launch_sweep_any(L, init, a, num_sms, s);
    if (!init && a.update == PA_UPDATE_HEATBATH) return launch_sweep_hb(L, a, num_sms, s);
#define PA_SWEEP_CASE(LL)                                                                      \
    case LL:                                                                                   \
        return init ? launch_sweep_t<LL, true, false>(a, num_sms, s) : launch_sweep_t<LL, false, false>(a, num_sms, s);
    switch (L) {
        PA_SWEEP_CASE(4)
        PA_SWEEP_CASE(8)
        PA_SWEEP_CASE(12)
        PA_SWEEP_CASE(16)
        PA_SWEEP_CASE(20)
        PA_SWEEP_CASE(24)
        PA_SWEEP_CASE(32)
        PA_SWEEP_CASE(40)
        PA_SWEEP_CASE(48)
        PA_SWEEP_CASE(64)
        PA_SWEEP_CASE(80)
        PA_SWEEP_CASE(96)
        PA_SWEEP_CASE(128)
        default:
            return cudaErrorInvalidValue;
    }
#undef PA_SWEEP_CASE
}

}  // namespace pa
