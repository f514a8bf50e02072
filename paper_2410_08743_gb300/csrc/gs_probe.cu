// gs_probe.cu - measured arithmetic peaks of the current GPU, the denominators
// of the "alu" roofline of the blending kernels (they are bound by FP32 and
// MUFU issue, not by memory), plus the FP64 FMA rate and the rate of global
// atomic adds (the backward blend's gradient atomics, the FP64 pose sums).
//
// Each probe is one wave of resident blocks running long unrolled loops of
// independent dependency chains, so that the pipe under test, not latency,
// limits it: scalar FFMA, paired FFMA (fma.rn.f32x2, both halves counted) and
// MUFU ex2 (each ex2 followed by one FADD to keep its argument bounded).  The
// rate per SM per cycle comes from clock64() readings (independent of the
// clock the GPU runs at): per SM, the work of its blocks over the span from
// its first block's start to its last block's end (the warp scheduler favours
// older warps, so the blocks of one SM finish at different times); the rate
// per second from CUDA events.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "gs_internal.cuh"

namespace gs {

#define PR_THREADS 256
#define PR_CHAINS 16
#define PR_ITERS 1024
#define PR_UNROLL 8
#define PR_FP64_DIV 16
#define PR_KINDS 4

__device__ __forceinline__ unsigned long long pr_pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float pr_sum2(unsigned long long r) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    return a + b;
}

// kind 0: FFMA; kind 1: fma.rn.f32x2; kind 2: ex2.approx + FADD; kind 3: DFMA
// (PR_ITERS / PR_FP64_DIV iterations: the FP64 rate is far below the FP32 one).
// cycles[3 * block + 0..2] = start clock, end clock, SM id
template <int KIND>
__global__ void __launch_bounds__(PR_THREADS) k_probe(float s, float* __restrict__ sink,
                                                      long long* __restrict__ cycles) {
    __syncthreads();
    const long long c0 = clock64();
    float acc = 0.0f;
    if (KIND == 0) {
        float x[PR_CHAINS];
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) x[c] = 1e-3f * (float)(threadIdx.x + c);
        for (int it = 0; it < PR_ITERS; it++) {
#pragma unroll
            for (int u = 0; u < PR_UNROLL; u++)
#pragma unroll
                for (int c = 0; c < PR_CHAINS; c++) x[c] = fmaf(x[c], s, 0.25f);
        }
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) acc += x[c];
    } else if (KIND == 1) {
        unsigned long long x[PR_CHAINS / 2];
        const unsigned long long sv = pr_pack(s, s), hv = pr_pack(0.25f, 0.25f);
#pragma unroll
        for (int c = 0; c < PR_CHAINS / 2; c++) x[c] = pr_pack(1e-3f * (float)(threadIdx.x + c), 1e-3f * (float)c);
        for (int it = 0; it < PR_ITERS; it++) {
#pragma unroll
            for (int u = 0; u < PR_UNROLL; u++)
#pragma unroll
                for (int c = 0; c < PR_CHAINS / 2; c++)
                    asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(sv), "l"(hv));
        }
#pragma unroll
        for (int c = 0; c < PR_CHAINS / 2; c++) acc += pr_sum2(x[c]);
    } else if (KIND == 3) {
        double x[PR_CHAINS];
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) x[c] = 1e-3 * (double)(threadIdx.x + c);
        const double sd = (double)s;
        for (int it = 0; it < PR_ITERS / PR_FP64_DIV; it++) {
#pragma unroll
            for (int u = 0; u < PR_UNROLL; u++)
#pragma unroll
                for (int c = 0; c < PR_CHAINS; c++) x[c] = fma(x[c], sd, 0.25);
        }
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) acc += (float)x[c];
    } else {
        float x[PR_CHAINS];
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) x[c] = -1e-4f * (float)(threadIdx.x + c);
        for (int it = 0; it < PR_ITERS; it++) {
#pragma unroll
            for (int u = 0; u < PR_UNROLL / 4; u++)
#pragma unroll
                for (int c = 0; c < PR_CHAINS; c++) {
                    float y;
                    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
                    x[c] = y - s;   // ex2 of a value in [-1, 0] lies in [0.5, 1]
                }
        }
#pragma unroll
        for (int c = 0; c < PR_CHAINS; c++) acc += x[c];
    }
    __syncthreads();
    const long long c1 = clock64();
    sink[(size_t)blockIdx.x * PR_THREADS + threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        cycles[3 * blockIdx.x] = c0;
        cycles[3 * blockIdx.x + 1] = c1;
        cycles[3 * blockIdx.x + 2] = (long long)smid;
    }
}

// lane operations one block of a probe executes
static double probe_lane_ops(int kind) {
    const double per_thread = kind == 2   ? (double)PR_ITERS * (PR_UNROLL / 4) * PR_CHAINS
                              : kind == 3 ? (double)(PR_ITERS / PR_FP64_DIV) * PR_UNROLL * PR_CHAINS
                                          : (double)PR_ITERS * PR_UNROLL * PR_CHAINS;
    return per_thread * PR_THREADS;
}

// Global atomic adds without a return value (red.global.add), every thread
// its own address per iteration, cycling through 2^PA_SLOT_BITS slots that
// stay resident in L2: scalar (VEC 1) or 16-byte vector (VEC 4) adds.
#define PA_THREADS 256
#define PA_ITERS 64
#define PA_SLOT_BITS 20
template <int VEC>
__global__ void __launch_bounds__(PA_THREADS) k_probe_red(float* __restrict__ buf) {
    const unsigned nthr = gridDim.x * blockDim.x;
    const unsigned mask = (1u << PA_SLOT_BITS) - 1u;
    unsigned slot = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < PA_ITERS; it++) {
        const unsigned k = slot & mask;
        if (VEC == 4) atomicAdd(reinterpret_cast<float4*>(buf) + k, make_float4(1.0f, 1.0f, 1.0f, 1.0f));
        else atomicAdd(buf + k, 1.0f);
        slot += nthr;
    }
}

}  // namespace gs

extern "C" int gs_measure_alu_peaks(int device, gs_alu_peaks* out) {
    using namespace gs;
    char msg[256];
    if (!out) return set_error(GS_EINVAL, "gs_measure_alu_peaks: out is NULL");
    *out = gs_alu_peaks{};
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "gs_measure_alu_peaks: cudaSetDevice(%d): %s", device, cudaGetErrorString(e));
        return set_error(GS_ECUDA, msg);
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per_sm[PR_KINDS] = {0, 0, 0, 0};
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_probe<0>, PR_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_probe<1>, PR_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], k_probe<2>, PR_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[3], k_probe<3>, PR_THREADS, 0);
    const int max_blocks = sms * *std::max_element(per_sm, per_sm + PR_KINDS);
    if (sms <= 0 || max_blocks <= 0) return set_error(GS_ECUDA, "gs_measure_alu_peaks: no resident blocks");
    float* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = GS_OK;
    double rate_clk[PR_KINDS] = {0, 0, 0, 0}, rate_s[PR_KINDS] = {0, 0, 0, 0}, mhz_sum = 0.0;
    double red_s[2] = {0, 0};
    float* abuf = nullptr;
    int mhz_n = 0;
    if ((e = cudaMalloc(&sink, sizeof(float) * (size_t)max_blocks * PR_THREADS)) != cudaSuccess ||
        (e = cudaMalloc(&cyc, sizeof(long long) * 3 * (size_t)max_blocks)) != cudaSuccess ||
        (e = cudaEventCreate(&ev0)) != cudaSuccess || (e = cudaEventCreate(&ev1)) != cudaSuccess) {
        snprintf(msg, sizeof(msg), "gs_measure_alu_peaks: setup: %s", cudaGetErrorString(e));
        rc = set_error(e == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA, msg);
    }
    std::vector<long long> hc(3 * (size_t)max_blocks);
    for (int kind = 0; kind < PR_KINDS && rc == GS_OK; kind++) {
        const int grid = sms * per_sm[kind];
        float best_ms = 0.0f;
        double best_clk = 0.0;
        for (int rep = 0; rep < 4 && rc == GS_OK; rep++) {   // the first repetition warms up
            cudaEventRecord(ev0, 0);
            if (kind == 0) k_probe<0><<<grid, PR_THREADS>>>(0.999f, sink, cyc);
            else if (kind == 1) k_probe<1><<<grid, PR_THREADS>>>(0.999f, sink, cyc);
            else if (kind == 2) k_probe<2><<<grid, PR_THREADS>>>(1.0f, sink, cyc);
            else k_probe<3><<<grid, PR_THREADS>>>(0.999f, sink, cyc);
            cudaEventRecord(ev1, 0);
            if ((e = cudaEventSynchronize(ev1)) != cudaSuccess ||
                (e = cudaMemcpy(hc.data(), cyc, sizeof(long long) * 3 * grid, cudaMemcpyDeviceToHost)) != cudaSuccess) {
                snprintf(msg, sizeof(msg), "gs_measure_alu_peaks: probe %d: %s", kind, cudaGetErrorString(e));
                rc = set_error(GS_ECUDA, msg);
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ev0, ev1);
            // per SM: its blocks' work over [first start, last end] (clock64 is per
            // SM; SM ids need not be dense, so the tables span the largest id seen)
            long long n_ids = 0;
            for (int b = 0; b < grid; b++) n_ids = std::max(n_ids, hc[3 * (size_t)b + 2] + 1);
            n_ids = std::min<long long>(n_ids, 4096);
            std::vector<long long> lo(n_ids, -1), hi(n_ids, -1);
            std::vector<int> nb(n_ids, 0);
            for (int b = 0; b < grid; b++) {
                const long long id = hc[3 * (size_t)b + 2];
                if (id < 0 || id >= n_ids) continue;
                const long long t0 = hc[3 * (size_t)b], t1 = hc[3 * (size_t)b + 1];
                if (nb[id] == 0 || t0 < lo[id]) lo[id] = t0;
                if (nb[id] == 0 || t1 > hi[id]) hi[id] = t1;
                nb[id]++;
            }
            std::vector<double> rates;
            double span_max = 0.0;
            for (long long id = 0; id < n_ids; id++) {
                if (nb[id] == 0 || hi[id] <= lo[id]) continue;
                rates.push_back(probe_lane_ops(kind) * nb[id] / (double)(hi[id] - lo[id]));
                span_max = std::max(span_max, (double)(hi[id] - lo[id]));
            }
            if (rates.empty()) {
                rc = set_error(GS_ECUDA, "gs_measure_alu_peaks: no block timings");
                break;
            }
            std::sort(rates.begin(), rates.end());
            const double clk = rates[rates.size() / 2];
            if (rep > 0 && (best_ms == 0.0f || ms < best_ms)) {
                best_ms = ms;
                best_clk = clk;
                mhz_sum += span_max / (ms * 1e3);   // longest SM span in cycles over the event time
                mhz_n++;
            }
        }
        rate_clk[kind] = best_clk;
        rate_s[kind] = best_ms > 0.0f ? probe_lane_ops(kind) * grid / (best_ms * 1e-3) : 0.0;
    }
    // atomic adds per second: a few waves of blocks, best of three timed runs
    if (rc == GS_OK) {
        const size_t bytes = sizeof(float4) << PA_SLOT_BITS;
        if ((e = cudaMalloc(&abuf, bytes)) != cudaSuccess || (e = cudaMemset(abuf, 0, bytes)) != cudaSuccess) {
            snprintf(msg, sizeof(msg), "gs_measure_alu_peaks: atomic buffer: %s", cudaGetErrorString(e));
            rc = set_error(e == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA, msg);
        }
        int per_sm_red = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_red, k_probe_red<4>, PA_THREADS, 0);
        const int grid = sms * std::max(1, per_sm_red) * 4;
        for (int v = 0; v < 2 && rc == GS_OK; v++) {
            float best_ms = 0.0f;
            for (int rep = 0; rep < 4 && rc == GS_OK; rep++) {   // the first repetition warms up
                cudaEventRecord(ev0, 0);
                if (v == 0) k_probe_red<1><<<grid, PA_THREADS>>>(abuf);
                else k_probe_red<4><<<grid, PA_THREADS>>>(abuf);
                cudaEventRecord(ev1, 0);
                if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) {
                    snprintf(msg, sizeof(msg), "gs_measure_alu_peaks: atomic probe %d: %s", v, cudaGetErrorString(e));
                    rc = set_error(GS_ECUDA, msg);
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, ev0, ev1);
                if (rep > 0 && (best_ms == 0.0f || ms < best_ms)) best_ms = ms;
            }
            red_s[v] = best_ms > 0.0f ? (double)grid * PA_THREADS * PA_ITERS / (best_ms * 1e-3) : 0.0;
        }
    }
    if (abuf) cudaFree(abuf);
    if (sink) cudaFree(sink);
    if (cyc) cudaFree(cyc);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (rc != GS_OK) return rc;
    out->sm_count = sms;
    out->probe_sm_mhz = mhz_n ? mhz_sum / mhz_n : 0.0;
    out->fp32_fma_per_sm_clk = rate_clk[0];
    out->fp32x2_fma_per_sm_clk = rate_clk[1];
    out->ex2_per_sm_clk = rate_clk[2];
    out->fp32_fma_per_s = rate_s[0];
    out->fp32x2_fma_per_s = rate_s[1];
    out->ex2_per_s = rate_s[2];
    out->fp64_fma_per_sm_clk = rate_clk[3];
    out->fp64_fma_per_s = rate_s[3];
    out->red_f32_per_s = red_s[0];
    out->red_f32x4_per_s = red_s[1];
    return GS_OK;
}
