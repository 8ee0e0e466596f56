// tile_io.cuh -- coalesced load/store of one bitsliced tile (1024 blocks).
#pragma once

#include <cstdint>

#include "internal.h"

namespace des3 {

// Lane `lane` of a tile holds the tile's blocks 64*(m/2) + 2*lane + (m%2),
// m = 0..31: each 16-byte access of the warp covers 512 contiguous bytes.
__device__ __forceinline__ void bs_load_tile(uint32_t (&w)[64], const uint8_t* base, uint32_t valid,
                                             bool vec, int lane) {
    if (vec && valid == kTileBlocks) {
        const uint4* src = reinterpret_cast<const uint4*>(base) + lane;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            uint4 v = __ldcs(src + 32 * j);
            w[2 * j] = v.x;
            w[32 + 2 * j] = v.y;
            w[2 * j + 1] = v.z;
            w[33 + 2 * j] = v.w;
        }
    } else {
        const uint2* src = reinterpret_cast<const uint2*>(base);
#pragma unroll
        for (int m = 0; m < 32; m++) {
            uint32_t blk = 64 * (m >> 1) + 2 * lane + (m & 1);
            uint2 v = make_uint2(0u, 0u);
            if (blk < valid) v = __ldcs(src + blk);
            w[m] = v.x;
            w[32 + m] = v.y;
        }
    }
}

__device__ __forceinline__ void bs_store_tile(const uint32_t (&w)[64], uint8_t* base, uint32_t valid,
                                              bool vec, int lane) {
    if (vec && valid == kTileBlocks) {
        uint4* dst = reinterpret_cast<uint4*>(base) + lane;
#pragma unroll
        for (int j = 0; j < 16; j++)
            __stcs(dst + 32 * j, make_uint4(w[2 * j], w[32 + 2 * j], w[2 * j + 1], w[33 + 2 * j]));
    } else {
        uint2* dst = reinterpret_cast<uint2*>(base);
#pragma unroll
        for (int m = 0; m < 32; m++) {
            uint32_t blk = 64 * (m >> 1) + 2 * lane + (m & 1);
            if (blk < valid) __stcs(dst + blk, make_uint2(w[m], w[32 + m]));
        }
    }
}

// w ^= the tile's bytes at base (same lane layout as bs_load_tile).
__device__ __forceinline__ void bs_xor_load_tile(uint32_t (&w)[64], const uint8_t* base, uint32_t valid,
                                                 bool vec, int lane) {
    if (vec && valid == kTileBlocks) {
        const uint4* src = reinterpret_cast<const uint4*>(base) + lane;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const uint4 v = __ldcs(src + 32 * j);
            w[2 * j] ^= v.x;
            w[32 + 2 * j] ^= v.y;
            w[2 * j + 1] ^= v.z;
            w[33 + 2 * j] ^= v.w;
        }
    } else {
        const uint2* src = reinterpret_cast<const uint2*>(base);
#pragma unroll
        for (int m = 0; m < 32; m++) {
            const uint32_t blk = 64 * (m >> 1) + 2 * lane + (m & 1);
            if (blk < valid) {
                const uint2 v = __ldcs(src + blk);
                w[m] ^= v.x;
                w[32 + m] ^= v.y;
            }
        }
    }
}

}  // namespace des3
