// Issue-rate probe of the SM pipes the search runs on: long independent
// chains of one instruction kind per thread, every SM filled, timed by the
// SM cycle counter.  It gives the measured denominator of the integer-pipe
// roofline (lane-operations per SM per clock) beside the derived one.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/tmd_probe.h"

namespace tmd {
namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CTAS_PER_SM = 8;

template <int OP>
__global__ void __launch_bounds__(PROBE_THREADS) k_pipe_probe(uint32_t* sink, uint32_t seed, int iters,
                                                              long long* cycles) {
    uint32_t a[PROBE_CHAINS];
    float f[PROBE_CHAINS];
    const uint32_t b = seed ^ threadIdx.x, c = seed * 3u + 7u;
    const float g = 1.0001f, h = 0.5f;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; i++) {
        a[i] = seed + (uint32_t)i * 0x9e3779b9u + threadIdx.x;
        f[i] = (float)(a[i] & 0xffffu);
    }
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; i++) {
            if (OP == 0) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
            if (OP == 1) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b), "r"(c));
            if (OP == 2) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
            if (OP == 3) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[i]) : "f"(g), "f"(h));
        }
    }
    const long long t1 = clock64();
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; i++) s ^= a[i] ^ __float_as_uint(f[i]);
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace tmd

extern "C" tmd_status tmd_pipe_rates(int device, double* out, int n_out) {
    using namespace tmd;
    if (!out || n_out < 1) return TMD_EINVAL;
    int ndev = 0, sms = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return TMD_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return TMD_ECUDA;
    const int ctas = sms * PROBE_CTAS_PER_SM, iters = 4096;
    uint32_t* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc((void**)&sink, (size_t)ctas * PROBE_THREADS * 4) != cudaSuccess) return TMD_ENOMEM;
    if (cudaMalloc((void**)&cyc, (size_t)ctas * 8) != cudaSuccess) {
        cudaFree(sink);
        return TMD_ENOMEM;
    }
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    tmd_status st = TMD_OK;
    std::vector<long long> h(ctas);
    double rates[4] = {0, 0, 0, 0}, mhz = 0;
    for (int op = 0; op < 4 && st == TMD_OK; op++) {
        for (int rep = 0; rep < 2 && st == TMD_OK; rep++) {  // the first run warms up
            cudaEventRecord(e0);
            switch (op) {
                case 0: k_pipe_probe<0><<<ctas, PROBE_THREADS>>>(sink, 12345u + rep, iters, cyc); break;
                case 1: k_pipe_probe<1><<<ctas, PROBE_THREADS>>>(sink, 12345u + rep, iters, cyc); break;
                case 2: k_pipe_probe<2><<<ctas, PROBE_THREADS>>>(sink, 12345u + rep, iters, cyc); break;
                default: k_pipe_probe<3><<<ctas, PROBE_THREADS>>>(sink, 12345u + rep, iters, cyc); break;
            }
            cudaEventRecord(e1);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaMemcpy(h.data(), cyc, (size_t)ctas * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
                st = TMD_ECUDA;
                break;
            }
            long long mx = 1;
            for (long long v : h) mx = v > mx ? v : mx;
            // lane-operations of the whole grid over the slowest CTA's cycles, per SM
            const double ops = (double)ctas * PROBE_THREADS * iters * PROBE_CHAINS;
            rates[op] = ops / ((double)sms * (double)mx);
            if (op == 0) mhz = (double)mx / (ms * 1e3);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    if (st != TMD_OK) return st;
    for (int i = 0; i < n_out && i < 4; i++) out[i] = rates[i];
    if (n_out > 4) out[4] = mhz;
    return TMD_OK;
}
