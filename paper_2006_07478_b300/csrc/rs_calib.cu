// rs_calib.cu -- a calibration kernel for the roofline of the region pipelines: the
// cascade's per-element arithmetic (three context-hash filters, Section 5's cascade of
// selective stages, with ballot compaction into a shared-memory queue between them and a
// count and sum at the end) over ONE region, with no region tags, work units, parent
// records or per-region outputs.  Its speed bounds from above what rs_tag_kernel and
// rs_pipeline_kernel can reach on the same elements: the difference is the cost of
// handling regions.  It is a measurement aid beside the pipeline, not part of it.
//
// Every warp is one processor with two queues of 256 items in shared memory (edges 1->2
// and 2->3).  It takes windows of 128 consecutive elements (4 per lane, one 16-byte
// load each, two windows loaded ahead) in a grid-stride order, filters them (node 1)
// into queue 1, and nodes 2 and 3 fire on full ensembles of 128 items as in the
// pipeline kernels (a node fires only when its output queue has room for an ensemble);
// the queues are drained with partial ensembles at the end.  Items in a queue carry no
// tag, so each slot position of the 4 is compacted by its own ballot.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rs_device.cuh"

namespace {

constexpr uint32_t CW = 128;   // items per ensemble
constexpr uint32_t CQ = 256;   // queue capacity (two ensembles)

struct CalibParams {
    const uint32_t *elements;
    unsigned long long n;
    uint32_t ctx;
    uint32_t c0s[3];     // per filter: c0 ^ (c0 >> 16), c0 = fmix32(salt ^ RS_GOLD)
    uint32_t theta[3];
    uint32_t m16, m19;   // 2^16 and 2^19 (kernel arguments, so they stay multiplies)
    unsigned long long *out;   // [count, sum]
};

// fmix32(x ^ c0): the first xor-shift distributes over the xor with c0; two right
// shifts are the high words of multiplies by 2^16 and 2^19
__device__ __forceinline__ uint32_t hash_c(uint32_t x, uint32_t c0s, uint32_t m16, uint32_t m19)
{
    uint32_t h = x ^ __umulhi(x, m16) ^ c0s;
    h *= 0x85EBCA6Bu;
    h ^= __umulhi(h, m19);
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// window w's 4 elements of this lane (zeros past n)
__device__ __forceinline__ uint4 load_window(const CalibParams &P, unsigned long long w, uint32_t lane, bool vec)
{
    const unsigned long long e = w * CW + 4u * lane;
    if (vec && e + 4 <= P.n) return ld_stream_v4(P.elements + e);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (e < P.n) v.x = __ldg(P.elements + e);
    if (e + 1 < P.n) v.y = __ldg(P.elements + e + 1);
    if (e + 2 < P.n) v.z = __ldg(P.elements + e + 2);
    if (e + 3 < P.n) v.w = __ldg(P.elements + e + 3);
    return v;
}

struct CalibWarp {
    const CalibParams &P;
    uint32_t lane, lt;
    uint32_t *q1, *q2;
    uint32_t h1 = 0, t1 = 0, h2 = 0, t2 = 0;
    uint32_t cnt = 0;
    unsigned long long sum = 0;

    __device__ CalibWarp(const CalibParams &p, uint32_t l, uint32_t *a, uint32_t *b)
        : P(p), lane(l), lt(lanemask_lt()), q1(a), q2(b) {}

    // append the kept items of the 4 slot positions to queue q at tail t
    __device__ __forceinline__ void push(uint32_t *q, uint32_t &t, const uint32_t (&y)[4], const bool (&k)[4])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t b = __ballot_sync(FULLMASK, k[i]);
            if (k[i]) q[(t + __popc(b & lt)) & (CQ - 1)] = y[i];
            t += __popc(b);
        }
    }

    // node 1 on window w (FULL: all of its 128 positions hold elements)
    template <bool FULL>
    __device__ __forceinline__ void node1(const uint4 v, unsigned long long w)
    {
        const uint32_t x[4] = {v.x, v.y, v.z, v.w};
        const unsigned long long e = w * CW + 4u * lane;
        bool k[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            k[i] = (FULL || e + i < P.n) && (hash_c(x[i], P.c0s[0], P.m16, P.m19) ^ P.ctx) < P.theta[0];
        push(q1, t1, x, k);
    }

    // node 2 on `take` items at the head of queue 1
    __device__ __forceinline__ void node2(uint32_t take)
    {
        uint32_t y[4];
        bool k[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t s = 32u * i + lane;
            y[i] = q1[(h1 + s) & (CQ - 1)];
            k[i] = s < take && (hash_c(y[i], P.c0s[1], P.m16, P.m19) ^ P.ctx) < P.theta[1];
        }
        __syncwarp();
        h1 += take;
        push(q2, t2, y, k);
        __syncwarp();
    }

    // node 3 on `take` items at the head of queue 2, folded into the count and sum
    __device__ __forceinline__ void node3(uint32_t take)
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t s = 32u * i + lane;
            const uint32_t z = q2[(h2 + s) & (CQ - 1)];
            const bool k = s < take && (hash_c(z, P.c0s[2], P.m16, P.m19) ^ P.ctx) < P.theta[2];
            cnt += k ? 1u : 0u;
            sum += k ? z : 0u;
        }
        __syncwarp();
        h2 += take;
    }

    // fire nodes 3 and 2 on full ensembles, downstream first, until queue 1 has room
    __device__ __forceinline__ void pump()
    {
        while (t1 - h1 >= CW) {
            while (t2 - h2 >= CW) node3(CW);
            node2(CW);
        }
        while (t2 - h2 >= CW) node3(CW);
    }

    __device__ __forceinline__ void drain()
    {
        while (t1 != h1) {
            while (t2 - h2 >= CW) node3(CW);
            node2(min(t1 - h1, CW));
        }
        while (t2 != h2) node3(min(t2 - h2, CW));
    }
};

__global__ void __launch_bounds__(256, 4) rs_calib_kernel(const __grid_constant__ CalibParams P)
{
    __shared__ uint32_t qs[8][2][CQ];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    CalibWarp C(P, lane, qs[warp][0], qs[warp][1]);
    const unsigned long long nwin = (P.n + CW - 1) / CW;
    const unsigned long long tw = (unsigned long long)gridDim.x * 8u;
    const bool vec = ((uintptr_t)P.elements & 15u) == 0;
    unsigned long long w = (unsigned long long)blockIdx.x * 8u + warp;
    uint4 v0 = w < nwin ? load_window(P, w, lane, vec) : make_uint4(0u, 0u, 0u, 0u);
    uint4 v1 = w + tw < nwin ? load_window(P, w + tw, lane, vec) : make_uint4(0u, 0u, 0u, 0u);
    for (; w < nwin; w += tw) {
        const uint4 cur = v0;
        v0 = v1;
        v1 = w + 2 * tw < nwin ? load_window(P, w + 2 * tw, lane, vec) : make_uint4(0u, 0u, 0u, 0u);
        if ((w + 1) * CW <= P.n) C.node1<true>(cur, w);
        else C.node1<false>(cur, w);
        __syncwarp();
        C.pump();
    }
    C.drain();
    const unsigned long long c = __reduce_add_sync(FULLMASK, C.cnt);
    const unsigned long long s = warp_sum_u64(C.sum);
    if (lane == 0 && c) {
        atomicAdd(P.out, c);
        atomicAdd(P.out + 1, s);
    }
}

}  // namespace

// Launch the calibration kernel on `stream` (out[0..1] must be zeroed first): a persistent
// grid of as many CTAs of 8 processors per SM as fit.  Returns the CUDA error code (0 on success).
int rs_launch_calib(const uint32_t *elements, unsigned long long n, uint32_t ctx, const uint32_t c0[3],
                    const uint32_t theta[3], unsigned long long *out, int n_sm, void *stream)
{
    CalibParams P;
    P.elements = elements;
    P.n = n;
    P.ctx = ctx;
    for (int i = 0; i < 3; ++i) {
        P.c0s[i] = c0[i] ^ (c0[i] >> 16);
        P.theta[i] = theta[i];
    }
    P.m16 = 1u << 16;
    P.m19 = 1u << 19;
    P.out = out;
    int bps = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, rs_calib_kernel, 256, 0);
    if (e != cudaSuccess) return (int)e;
    if (bps < 1) bps = 1;
    rs_calib_kernel<<<bps * n_sm, 256, 0, (cudaStream_t)stream>>>(P);
    return (int)cudaGetLastError();
}
