// Host build of the library's integer FP64 <-> FP32 conversions, for the CPU
// tests that compare them with the host's own IEEE conversions.
#include "conv.cuh"

extern "C" void conv_narrow(const uint64_t *in, uint32_t *out, long n) {
    for (long i = 0; i < n; i++) out[i] = mds::f64_to_f32_bits(in[i]);
}

extern "C" void conv_widen(const uint32_t *in, uint64_t *out, long n) {
    for (long i = 0; i < n; i++) out[i] = mds::f32_to_f64_bits(in[i]);
}
