// lp_stage_big.cuh -- visit-order ranks of an LP larger than a warp's one-word-per-lane
// key bitmap, for the large-LP kernels of the 3-D and d-dimensional solvers.
//
// The visit order is the key order of the Feistel network of lp2d_device.cuh (Sec. 2.1
// asks for a random order).  A warp marks every key in a bitmap of the key domain
// (4^h bits; several words per lane), turns the word counts into prefix counts, and
// hands each constraint to the caller with its rank, the number of smaller keys.
#pragma once

#include "lp2d_device.cuh"
#include "lp2d_staged.cuh"

namespace lp2d {

// Words of the key bitmap of an LP with m constraints: max(1, 4^h / 32).
__device__ __forceinline__ int key_words(const VisitOrder& vo) {
    const uint64_t dom = vo.domain();
    return dom >= 32 ? static_cast<int>(dom >> 5) : 1;
}

// One warp: bm and pre hold key_words(vo) words each (the caller sizes them for its
// largest LP); copy(rank, q) is called once for every constraint q < m, from the lane
// that handles q.  bm keeps the LP's key bitmap afterwards.  Completion: the copies'
// own (cp_async_wait_all) then __syncwarp.
template <typename Copy>
__device__ __forceinline__ void stage_ranks_warp(const VisitOrder& vo, int m, unsigned* bm, int* pre, int lane,
                                                 Copy copy) {
    const int nwords = key_words(vo);
    for (int w = lane; w < nwords; w += 32) bm[w] = 0u;
    __syncwarp();
    for (int q = lane; q < m; q += 32) {
        const uint32_t e = vo.enc(static_cast<uint32_t>(q));
        atomicOr(bm + (e >> 5), 1u << (e & 31u));
    }
    __syncwarp();
    // lane l owns words l K .. l K + K - 1
    const int K = (nwords + 31) / 32;
    int local = 0;
    for (int i = 0; i < K; ++i) {
        const int w = lane * K + i;
        if (w < nwords) local += __popc(bm[w]);
    }
    int run = warp_inclusive_scan(local, lane) - local;
    for (int i = 0; i < K; ++i) {
        const int w = lane * K + i;
        if (w < nwords) {
            pre[w] = run;
            run += __popc(bm[w]);
        }
    }
    __syncwarp();
    for (int q = lane; q < m; q += 32) {
        const uint32_t e = vo.enc(static_cast<uint32_t>(q));
        const int wi = static_cast<int>(e >> 5);
        copy(pre[wi] + __popc(bm[wi] & ((1u << (e & 31u)) - 1u)), q);
    }
}

}  // namespace lp2d
