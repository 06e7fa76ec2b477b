// mesh.h -- launchers of mesh.cu (zero crossings, marching cubes, G-GPDF training set).
#pragma once

#include "internal.h"

namespace vgp {

// read-only view of the fused global grid: leaf hash table, pool index per slot, per-leaf
// known-voxel bitmask (8 words) and FP64 values (512 per leaf)
struct GridView {
    const uint64_t* keys;
    uint32_t mask;
    const int32_t* slot2pool;
    const unsigned long long* known;
    const double* D;
    const double* C = nullptr;  // fused properties [pool][512][nc] and variances (NaN: none)
    const double* W = nullptr;
    int nc = 0;
};

// 256 x 16 table of cell-local edges (5 triangles at most) and the triangle count per mask
void build_mc_table(uint8_t* tab, uint8_t* ntri);

// leaves of the grid (all, or those the latest fusion touched): pool index and key
void mesh_leaf_list(const GridView& g, const int32_t* flags, int active_only, int32_t* lpool, uint64_t* lkey,
                    int* count, cudaStream_t st);
// count pass (emit = false: cnt[leaf]) and emit pass (segments at base + off[leaf])
// xprop / vprop (may be null): interpolated fused properties [n][g.nc] / [T][3][g.nc]
void mesh_crossings(const GridView& g, const int32_t* lpool, const uint64_t* lkey, int nl, double vs, int64_t* cnt,
                    const int64_t* off, int64_t base, float* xyz, uint64_t* owner, uint8_t* slot, double* xprop,
                    bool emit, cudaStream_t st);
void mesh_triangles(const GridView& g, const int32_t* lpool, const uint64_t* lkey, int nl, const uint8_t* tab,
                    const uint8_t* ntri, double vs, int64_t* cnt, const int64_t* off, double* xyz, uint64_t* ekey,
                    uint8_t* eaxis, double* vprop, bool emit, cudaStream_t st);
// training-set update: keep[i] = 0 for points in leaves the latest fusion touched
void store_keep(const float* pts, int64_t n, double vs, const GridView& g, const int32_t* flags, int64_t* keep,
                cudaStream_t st);
void store_compact(const float* pts, int64_t n, const int64_t* keep, const int64_t* pos, float* out,
                   cudaStream_t st);

}  // namespace vgp
