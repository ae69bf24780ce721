// pa_sweep_hb.cu -- step 3 with the heatbath update (Sec. IV): the instantiations of the
// fused sweep kernel of pa_sweep.cuh for every supported L, in a translation unit of their
// own so that the two updates compile in parallel.
#include "pa_sweep.cuh"

namespace pa {

cudaError_t launch_sweep_hb(int L, const SweepArgs &a, int num_sms, cudaStream_t s)
{
    switch (L) {
        case 4: return launch_sweep_t<4, false, true>(a, num_sms, s);
        case 8: return launch_sweep_t<8, false, true>(a, num_sms, s);
        case 12: return launch_sweep_t<12, false, true>(a, num_sms, s);
        case 16: return launch_sweep_t<16, false, true>(a, num_sms, s);
        case 20: return launch_sweep_t<20, false, true>(a, num_sms, s);
        case 24: return launch_sweep_t<24, false, true>(a, num_sms, s);
        case 32: return launch_sweep_t<32, false, true>(a, num_sms, s);
        case 40: return launch_sweep_t<40, false, true>(a, num_sms, s);
        case 48: return launch_sweep_t<48, false, true>(a, num_sms, s);
        case 64: return launch_sweep_t<64, false, true>(a, num_sms, s);
        case 80: return launch_sweep_t<80, false, true>(a, num_sms, s);
        case 96: return launch_sweep_t<96, false, true>(a, num_sms, s);
        case 128: return launch_sweep_t<128, false, true>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pa
