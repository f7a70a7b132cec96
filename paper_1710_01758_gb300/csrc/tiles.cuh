// Shared-memory tile layouts of the column-transform kernels (q = A p and the right-hand side):
// 16-column coil tiles written by TMA with the 128-byte swizzle, the padded per-column exchange
// regions of the transforms, and the row addressing of a thread's 16 values.
#pragma once

#include "kernels.h"
#include "tma.cuh"

namespace sb {
namespace tiles {

constexpr int TX = kColTile;

// bytes to skip from `p` (shared memory) to the next 1024-byte boundary of the shared window
// (the 128-byte TMA swizzle repeats every 1024 bytes); indexing the shared symbol itself keeps
// the accesses in the shared address space
__device__ __forceinline__ uint32_t pad_to_1024(const void* p) {
    return (1024u - (smem_addr(p) & 1023u)) & 1023u;
}

// float2 index of element (row, col) of a [rows][16] complex tile written by TMA with the
// 128-byte swizzle (16-byte chunk index XOR row % 8)
__device__ __forceinline__ int swz(int row, int col) {
    return row * TX + ((((col >> 1) ^ (row & 7)) << 1) | (col & 1));
}

// positions of one column transform in its exchange region, plus the per-column stride
template <int NY>
struct ExIdx {
    static constexpr int kStride = ((NY + NY / 16 + 7) / 16) * 16 + 8;  // >= NY + NY/16, = 8 mod 16
    int base;
    __device__ __forceinline__ int operator()(int pos) const { return base + pos + (pos >> 4); }
};

// Row t + T e of a thread's column in a swizzled tile: when T is a multiple of 8 the swizzle
// term depends on t only, so the 16 rows sit at constant offsets from one base index.
template <int T>
struct TileRows {
    int base, col, t;
    __device__ __forceinline__ TileRows(int t_, int col_) : base(swz(t_, col_)), col(col_), t(t_) {}
    __device__ __forceinline__ int operator()(int e) const {
        if constexpr (T % 8 == 0) return base + e * T * TX;
        else return swz(t + T * e, col);
    }
};

}  // namespace tiles
}  // namespace sb
