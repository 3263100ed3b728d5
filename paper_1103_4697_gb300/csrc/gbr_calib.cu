// Arithmetic ceilings of the library's modular arithmetic on this GPU.
//
// Each thread runs CHAINS independent Montgomery chains so the integer pipes,
// not latency, limit throughput.  The per-chain constants depend on the thread
// id so the compiler cannot fold them; the final value is stored so nothing is
// dead code.
#include "gbr_core.h"

namespace gbr {

template <int CHAINS, int KIND>
__global__ void k_calib(const ModP *mods, int iters, uint32_t *sink) {
    const ModP M = mods[threadIdx.x & 15];
    uint32_t x[CHAINS], y[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
        x[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % M.p;
        y[c] = (threadIdx.x * 31u + c * 17u + 3u) % M.p;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            if (KIND == 2)
                x[c] = mp_fma3(x[c], y[c], y[(c + 1) % CHAINS], x[(c + 3) % CHAINS], y[(c + 5) % CHAINS],
                               x[(c + 6) % CHAINS], M);
            else if (KIND == 1)
                x[c] = mp_mulsub(x[c], y[c], y[(c + 1) % CHAINS], x[(c + 3) % CHAINS], M);
            else
                x[c] = mp_mul(x[c], y[c], M);
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc ^= x[c];
    if (acc == 0x12345678u) sink[0] = acc;
}

}  // namespace gbr

using namespace gbr;

extern "C" int gbr_calibrate(gbr_ctx *c, gbr_calib *out) {
    if (!c || !out) return GBR_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    int sms = 1, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, c->device);
    uint32_t *sink = (uint32_t *)c->dalloc(64);
    if (!sink) return c->fail(GBR_ENOMEM, "calibration scratch");
    const int block = 256, grid = sms * 8, iters = 4096;
    const int CH = 8;
    double rates[3];
    cudaError_t e = cudaSuccess;
    for (int fused = 0; fused < 3 && e == cudaSuccess; ++fused) {
        auto launch = [&]() {
            if (fused == 2) k_calib<CH, 2><<<grid, block, 0, c->stream>>>(c->d_mods, iters, sink);
            else if (fused == 1) k_calib<CH, 1><<<grid, block, 0, c->stream>>>(c->d_mods, iters, sink);
            else k_calib<CH, 0><<<grid, block, 0, c->stream>>>(c->d_mods, iters, sink);
        };
        launch();   // warm-up
        cudaEventRecord(c->ev[6], c->stream);
        const int reps = 5;
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(c->ev[7], c->stream);
        e = cudaEventSynchronize(c->ev[7]);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]);
        rates[fused] = (double)grid * block * iters * CH * reps / (ms * 1e-3);
    }
    c->dfree(sink);
    if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "calibration", e);
    out->modmul_per_s = rates[0];
    out->mulsub_per_s = rates[1];
    out->fma3_per_s = rates[2];
    out->sm_clock_mhz = clk / 1000.0;
    out->sms = sms;
    return GBR_OK;
}
