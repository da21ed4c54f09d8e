// Phase-timing build of the kernels (a profiling tool, not part of libccl.so).  With
// CCL_PHASE_TIMING defined, the kernel bodies call ccl_phase_tick at every phase barrier;
// thread 0 of each CTA adds the clock64 cycles since its previous tick to a per-(kernel,
// phase) sum.  The sums give each phase's share of a CTA's time.  Built and driven by
// paper_1606_05973_gb300/phase_timing.py.
#include "ccl_kernels.cu"

namespace ccl {

__device__ unsigned long long g_phase_cycles[3][16];

__device__ void ccl_phase_tick(int kernel, int phase, int tid)
{
    __shared__ long long s_prev;
    if (tid != 0)
        return;
    const long long now = clock64();
    if (phase > 0)
        atomicAdd(&g_phase_cycles[kernel][phase - 1], (unsigned long long)(now - s_prev));
    s_prev = now;
}

}  // namespace ccl

// summed cycles, [kernel][phase] with kernel 0 = tile pass, 1 = global, 2 = final
extern "C" int ccl_phase_read(unsigned long long *out)
{
    return (int)cudaMemcpyFromSymbol(out, ccl::g_phase_cycles, sizeof(ccl::g_phase_cycles));
}

extern "C" int ccl_phase_reset(void)
{
    static const unsigned long long zero[3 * 16] = {};
    return (int)cudaMemcpyToSymbol(ccl::g_phase_cycles, zero, sizeof(zero));
}
