// Nearest-neighbour matching of BRIEF / RRIEF descriptors for sm_103a
// (Sec. 2.1 (e): descriptors are matched by nearest neighbour).
//
// One warp per query descriptor of set A.  The 32 lanes stride over set B;
// each lane keeps its best and second-best candidate as 64-bit keys
// (distance << 32 | index), so ties fall to the lower index and the warp's
// two best are found with a butterfly of shuffles that merges (best, second)
// pairs.
//   BRIEF: distance = popc(a ^ b), the Hamming distance of the 64-bit words.
//   RRIEF: distance = sum_k (a_k - b_k)^2 over the 64 ranks (bytes), computed
//          as |a|^2 + |b|^2 - 2 a.b with exact integer __dp4a on the packed
//          bytes (at most 64 * 255^2, well inside 32 bits).
#include <climits>

#include "common.cuh"

namespace sift3d {

namespace {

constexpr int MATCH_WARPS = 8;   // queries per CTA
constexpr unsigned long long kNone = ~0ull;

__device__ __forceinline__ unsigned long long key_of(unsigned dist, int idx) {
    return ((unsigned long long)dist << 32) | (unsigned)idx;
}

__device__ __forceinline__ void keep(unsigned long long k, unsigned long long& b1, unsigned long long& b2) {
    if (k < b1) {
        b2 = b1;
        b1 = k;
    } else if (k < b2) {
        b2 = k;
    }
}

template <int KIND>
__global__ void __launch_bounds__(32 * MATCH_WARPS) match_kernel(const MatchArgs a) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * MATCH_WARPS + (threadIdx.x >> 5);
    if (q >= a.na) return;   // whole warps leave together
    unsigned long long b1 = kNone, b2 = kNone;
    if constexpr (KIND == SIFT3D_DESC_BRIEF) {
        const uint64_t* A = static_cast<const uint64_t*>(a.a);
        const uint64_t* B = static_cast<const uint64_t*>(a.b);
        const uint64_t qa = A[q];
        for (int j = lane; j < a.nb; j += 32) keep(key_of((unsigned)__popcll(qa ^ B[j]), j), b1, b2);
    } else {
        // 64 ranks = 16 words of 4 bytes
        const uint4* A = static_cast<const uint4*>(a.a);
        const uint4* B = static_cast<const uint4*>(a.b);
        uint4 qa[4];
        unsigned qq = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            qa[w] = A[(int64_t)q * 4 + w];
            qq = __dp4a(qa[w].x, qa[w].x, qq);
            qq = __dp4a(qa[w].y, qa[w].y, qq);
            qq = __dp4a(qa[w].z, qa[w].z, qq);
            qq = __dp4a(qa[w].w, qa[w].w, qq);
        }
        for (int j = lane; j < a.nb; j += 32) {
            unsigned dot = 0, cc = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint4 c = B[(int64_t)j * 4 + w];
                dot = __dp4a(qa[w].x, c.x, dot);
                dot = __dp4a(qa[w].y, c.y, dot);
                dot = __dp4a(qa[w].z, c.z, dot);
                dot = __dp4a(qa[w].w, c.w, dot);
                cc = __dp4a(c.x, c.x, cc);
                cc = __dp4a(c.y, c.y, cc);
                cc = __dp4a(c.z, c.z, cc);
                cc = __dp4a(c.w, c.w, cc);
            }
            keep(key_of(qq + cc - 2u * dot, j), b1, b2);
        }
    }
    // merge the lanes' (best, second) pairs
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, b1, off);
        const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, b2, off);
        const unsigned long long lo = b1 < o1 ? b1 : o1;
        const unsigned long long hi = b1 < o1 ? o1 : b1;
        const unsigned long long s = b2 < o2 ? b2 : o2;
        b1 = lo;
        b2 = hi < s ? hi : s;
    }
    if (lane == 0) {
        a.nn[q] = b1 == kNone ? -1 : (int)(b1 & 0xffffffffu);
        a.dist[q] = b1 == kNone ? INT_MAX : (int)(b1 >> 32);
        if (a.dist2 != nullptr) a.dist2[q] = b2 == kNone ? INT_MAX : (int)(b2 >> 32);
    }
}

}  // namespace

LaunchSpec match_spec(int kind, const MatchArgs& a) {
    LaunchSpec s;
    if (kind == SIFT3D_DESC_BRIEF) s.func = reinterpret_cast<const void*>(&match_kernel<SIFT3D_DESC_BRIEF>);
    else if (kind == SIFT3D_DESC_RRIEF) s.func = reinterpret_cast<const void*>(&match_kernel<SIFT3D_DESC_RRIEF>);
    else return s;
    s.grid = dim3((unsigned)((a.na + MATCH_WARPS - 1) / MATCH_WARPS));
    s.block = dim3(32 * MATCH_WARPS);
    s.smem = 0;
    s.name = "match";
    return s;
}

}  // namespace sift3d
