// Arithmetic ceilings of the library's modular arithmetic on this GPU.
//
// Each thread runs CHAINS independent chains: chain c reads only its own value
// and loop-invariant multipliers, so with enough chains per thread the integer
// pipes, not latency, limit throughput (the host keeps the best rate over
// several chain counts, which shows where the rate stops rising).  The
// multipliers depend on the thread id so the compiler cannot fold them; the
// final values are combined and stored so nothing is dead code.
#include "gbr_core.h"

namespace gbr {

enum CalibKind { CAL_MUL = 0, CAL_MULSUB = 1, CAL_FMA3 = 2, CAL_SHOUP = 3 };

template <int CHAINS, int KIND>
__global__ void k_calib(const ModP *mods, int iters, uint32_t *sink) {
    const ModP M = mods[threadIdx.x & 15];
    uint32_t x[CHAINS], y[CHAINS + 3];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % M.p;
#pragma unroll
    for (int c = 0; c < CHAINS + 3; ++c) y[c] = (threadIdx.x * 31u + c * 17u + 3u) % M.p;
    // Shoup form of the multiplier y[c]: floor(y 2^32 / p)
    uint32_t yp[KIND == CAL_SHOUP ? CHAINS : 1];
#pragma unroll
    for (int c = 0; c < (KIND == CAL_SHOUP ? CHAINS : 1); ++c) yp[c] = (uint32_t)(((uint64_t)y[c] << 32) / M.p);
    const uint32_t np = 0u - M.p;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            if (KIND == CAL_FMA3)
                x[c] = mp_fma3(x[c], y[c], y[c + 1], x[c], y[c + 2], x[c], M);
            else if (KIND == CAL_MULSUB)
                x[c] = mp_mulsub(x[c], y[c], y[c + 1], x[c], M);
            else if (KIND == CAL_SHOUP)   // one Horner step acc y + c with a fixed multiplier (no reduction)
                x[c] = __umulhi(x[c], yp[c]) * np + (x[c] * y[c] + y[c + 1]);
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
    // operations per second of each kind, best over 4, 8 and 16 chains per thread
    double rates[4] = {0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int kind = 0; kind < 4 && e == cudaSuccess; ++kind)
        for (int ch : {4, 8, 16}) {
            auto launch = [&]() {
#define GBR_CAL(K)                                                                                   \
    if (ch == 4) k_calib<4, K><<<grid, block, 0, c->stream>>>(c->d_mods, iters, sink);               \
    else if (ch == 8) k_calib<8, K><<<grid, block, 0, c->stream>>>(c->d_mods, iters, sink);          \
    else k_calib<16, K><<<grid, block, 0, c->stream>>>(c->d_mods, iters, sink);
                if (kind == CAL_FMA3) { GBR_CAL(CAL_FMA3) }
                else if (kind == CAL_MULSUB) { GBR_CAL(CAL_MULSUB) }
                else if (kind == CAL_SHOUP) { GBR_CAL(CAL_SHOUP) }
                else { GBR_CAL(CAL_MUL) }
#undef GBR_CAL
            };
            launch();   // warm-up
            cudaEventRecord(c->ev[6], c->stream);
            const int reps = 5;
            for (int r = 0; r < reps; ++r) launch();
            cudaEventRecord(c->ev[7], c->stream);
            e = cudaEventSynchronize(c->ev[7]);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]);
            if (e != cudaSuccess) break;
            rates[kind] = std::max(rates[kind], (double)grid * block * iters * ch * reps / (ms * 1e-3));
        }
    c->dfree(sink);
    if (e != cudaSuccess) return c->fail(GBR_EDEVICE, "calibration", e);
    out->modmul_per_s = rates[CAL_MUL];
    out->mulsub_per_s = rates[CAL_MULSUB];
    out->fma3_per_s = rates[CAL_FMA3];
    out->shoup_per_s = rates[CAL_SHOUP];
    out->sm_clock_mhz = clk / 1000.0;
    out->sms = sms;
    return GBR_OK;
}
