// Device helpers of the exact parametric search (Section 2.1): the capacity
// line of a cut, and the problem restricted to the pixels between two nested
// cuts, scaled to integers at a rational lambda.
//
// For a source set S (mask 1 = s side) the cut of Section 2 costs
//   cap_S(lambda) = sum_{p not in S} cs(p, lambda) + sum_{p in S} ct(p)
//                 + sum over neighbour pairs (p in S, q not in S) of w(p, q)
// and with cs = src0 + slope * lambda this is a line a_S + b_S * lambda,
//   a_S = sum_{p not in S} src0(p) + sum_{p in S} ct(p) + cut pair capacities,
//   b_S = sum_{p not in S} slope(p).
// The minimum cut value F(lambda) is the lower envelope of these lines; its
// breakpoints are where the lines of consecutive maximal cuts cross.
//
// Between two maximal cuts S1 (optimal at lambda_1) and S2 (optimal at
// lambda_2 > lambda_1) every maximal cut for lambda in [lambda_1, lambda_2]
// lies between them (the cuts are nested).  Fixing S1 to the s side and the
// complement of S2 to the t side leaves a problem on D = S2 \ S1 alone: a pixel
// d of D keeps its pair arcs to other pixels of D, its arcs from S1 become part
// of its source arc and its arcs into the complement of S2 part of its sink
// arc.  Every cut between S1 and S2 costs a constant plus that problem's cut,
// so its maximal source set, joined with S1, is the maximal cut of the whole
// problem.  At lambda = p / q all capacities of the restricted problem are
// multiplied by q, which keeps them integer.
#include <cstdint>

#include "pmf.h"
#include "pmf_internal.h"

using namespace pmf;

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of v, added to *out by one atomic (integer: the order of the
// additions does not change the result)
__device__ void block_add(long long v, unsigned long long *out) {
    __shared__ long long part[kThreads / 32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        long long s = lane < kThreads / 32 ? part[lane] : 0;
        s = warp_sum(s);
        if (lane == 0 && s) atomicAdd(out, (unsigned long long)s);
    }
    __syncthreads();
}

// one block row per mask (blockIdx.y); pixels strided over blockIdx.x
__global__ void __launch_bounds__(kThreads) cut_lines_kernel(int H, int W, const int32_t *w_h, const int32_t *w_v,
                                                             const int32_t *src0, const int32_t *slope,
                                                             const int32_t *sink, const uint8_t *base,
                                                             const uint8_t *masks, uint8_t *uni,
                                                             unsigned long long *lines) {
    const int k = blockIdx.y;
    const size_t N = (size_t)H * W;
    const uint8_t *M = masks + (size_t)k * N;
    auto in_s = [&](size_t i) -> bool { return M[i] != 0 || (base != nullptr && base[i] != 0); };
    long long a = 0, b = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const bool s = in_s(i);
        if (uni) uni[(size_t)k * N + i] = s ? 1 : 0;
        if (!s) {
            a += src0[i];
            b += slope[i];
            continue;
        }
        a += sink[i];
        // pair arcs from this s-side pixel to t-side neighbours
        if (x + 1 < W && !in_s(i + 1)) a += w_h[i];
        if (x > 0 && !in_s(i - 1)) a += w_h[i - 1];
        if (y + 1 < H && !in_s(i + W)) a += w_v[i];
        if (y > 0 && !in_s(i - W)) a += w_v[i - W];
    }
    block_add(a, lines + 2 * k);
    block_add(b, lines + 2 * k + 1);
}

// the restricted problem on D = S2 \ S1, scaled by q at lambda = p / q; sums:
// [0] sum of its source capacities, [1] sum of its sink capacities over D,
// [2] pixels with capacities out of range, [3] pixels in D
__global__ void __launch_bounds__(kThreads) restrict_kernel(int H, int W, const int32_t *w_h, const int32_t *w_v,
                                                            const int32_t *src0, const int32_t *slope,
                                                            const int32_t *sink, const uint8_t *s1,
                                                            const uint8_t *s2, long long p, long long q,
                                                            int32_t *wh_o, int32_t *wv_o, int32_t *src_o,
                                                            int32_t *sink_o, unsigned long long *sums) {
    const size_t N = (size_t)H * W;
    auto in_d = [&](size_t i) -> bool { return s2[i] != 0 && s1[i] == 0; };
    long long scs = 0, sct = 0, bad = 0, nd = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        // a pixel outside D gets no arcs but a unit sink arc: with no source
        // arc it carries no flow and costs nothing on the t side, and it can
        // reach t, so the maximal source set never contains it
        long long cs = 0, ct = 1, wr = 0, wd = 0;
        if (in_d(i)) {
            ++nd;
            long long from_s1 = 0, to_out = 0;   // pair capacities to fixed neighbours
            auto nb = [&](size_t j, long long w) {
                if (s1[j]) from_s1 += w;
                else if (!s2[j]) to_out += w;
            };
            if (x + 1 < W) nb(i + 1, w_h[i]);
            if (x > 0) nb(i - 1, w_h[i - 1]);
            if (y + 1 < H) nb(i + W, w_v[i]);
            if (y > 0) nb(i - W, w_v[i - W]);
            cs = q * ((long long)src0[i] + from_s1) + p * (long long)slope[i];
            ct = q * ((long long)sink[i] + to_out);
            wr = (x + 1 < W && in_d(i + 1)) ? q * (long long)w_h[i] : 0;
            wd = (y + 1 < H && in_d(i + W)) ? q * (long long)w_v[i] : 0;
            if (cs < 0 || cs > PMF_INF || ct < 0 || ct > PMF_INF || wr > PMF_MAX_PAIRWISE || wd > PMF_MAX_PAIRWISE)
                ++bad;
            scs += cs;
            sct += ct;
        }
        const bool ok = cs >= 0 && cs <= PMF_INF && ct >= 0 && ct <= PMF_INF && wr <= PMF_MAX_PAIRWISE &&
                        wd <= PMF_MAX_PAIRWISE;
        src_o[i] = ok ? (int32_t)cs : 0;
        sink_o[i] = ok ? (int32_t)ct : 0;
        wh_o[i] = ok ? (int32_t)wr : 0;
        wv_o[i] = ok ? (int32_t)wd : 0;
    }
    block_add(scs, sums + 0);
    block_add(sct, sums + 1);
    block_add(bad, sums + 2);
    block_add(nd, sums + 3);
}

int blocks_for(size_t n) {
    const size_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 1184 ? 1184 : b));
}

}  // namespace

extern "C" PMF_API pmf_status pmf_cut_lines(int32_t H, int32_t W, const int32_t *w_h, const int32_t *w_v,
                                            const int32_t *src0, const int32_t *slope, const int32_t *sink,
                                            const uint8_t *base, const uint8_t *masks, int32_t n_masks,
                                            uint8_t *union_out, int64_t *lines, void *cuda_stream) {
    if (H < 1 || W < 1 || n_masks < 1 || n_masks > 65535 || !w_h || !w_v || !src0 || !slope || !sink || !masks ||
        !lines)
        return PMF_ERR_INVALID_ARG;
    if ((int64_t)H * W > (1 << 28)) return PMF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(lines, 0, sizeof(int64_t) * 2 * (size_t)n_masks, s);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_cut_lines: clear");
    (void)cudaGetLastError();
    const dim3 grid(blocks_for((size_t)H * W), n_masks);
    cut_lines_kernel<<<grid, kThreads, 0, s>>>(H, W, w_h, w_v, src0, slope, sink, base, masks, union_out,
                                               reinterpret_cast<unsigned long long *>(lines));
    return cuda_err_at(cudaGetLastError(), "pmf_cut_lines: launch");
}

extern "C" PMF_API pmf_status pmf_restrict_between(int32_t H, int32_t W, const int32_t *w_h, const int32_t *w_v,
                                                   const int32_t *src0, const int32_t *slope,
                                                   const int32_t *sink, const uint8_t *s1, const uint8_t *s2,
                                                   int64_t p, int64_t q, int32_t *w_h_out, int32_t *w_v_out,
                                                   int32_t *src0_out, int32_t *sink_out, int64_t *sums,
                                                   void *cuda_stream) {
    if (H < 1 || W < 1 || !w_h || !w_v || !src0 || !slope || !sink || !s1 || !s2 || !w_h_out || !w_v_out ||
        !src0_out || !sink_out || !sums)
        return PMF_ERR_INVALID_ARG;
    if ((int64_t)H * W > (1 << 28)) return PMF_ERR_INVALID_ARG;
    // |p|, q bounded so that no product of a capacity (< 2^31) overflows int64
    if (q < 1 || q > (1LL << 31) || p < 0 || p > (1LL << 31)) return PMF_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(int64_t) * 4, s);
    if (e != cudaSuccess) return cuda_err_at(e, "pmf_restrict_between: clear");
    (void)cudaGetLastError();
    restrict_kernel<<<blocks_for((size_t)H * W), kThreads, 0, s>>>(
        H, W, w_h, w_v, src0, slope, sink, s1, s2, p, q, w_h_out, w_v_out, src0_out, sink_out,
        reinterpret_cast<unsigned long long *>(sums));
    return cuda_err_at(cudaGetLastError(), "pmf_restrict_between: launch");
}
