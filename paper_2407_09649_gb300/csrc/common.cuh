// common.cuh -- device-side definitions shared by the CUDA translation units.
//
// Keys, hashing, voxel indexing (Sec. IV-A voxelisation into 8^3-voxel leaves, Sec. III-B),
// per-query status codes and the run-time parameters of the GP (Sec. III-A).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vgpdf.h"

namespace vgp {

constexpr uint64_t kEmpty = ~0ull;          // empty hash slot
constexpr int64_t kKeyBias = 1ll << 20;      // 21-bit biased coordinate fields
constexpr double kIjkLimit = 1048512.0;      // |ijk| < 2^20 - 64 keeps +-1 leaf neighbours valid

// device error bits (OR-ed into the map's error word)
enum : int {
    kErrTableFull = 1,
    kErrTimeout = 2,
    kErrCapacity = 4,   // an internal buffer bound was exceeded
    kErrFactor = 8,
    kErrLaunch = 16,    // a graph capture, instantiation or launch failed
    kErrAlloc = 32      // a solve workspace could not be allocated (nothing was launched)
};

// Run-time parameters, expanded once on the host.
struct DevParams {
    double vs;          // voxel size
    double l, l2;       // length scale and its square
    double inv2l2;      // 1 / (2 l^2)
    double s2;          // sigma_occ^2
    double d_max;
    double log_floor;   // -d_max^2 / (2 l^2)
    double d_var_floor;
    float inv2l2_log2e; // log2(e) / (2 l^2), for exp2f of the FP32 path
    float inv2l2_hi, inv2l2_lo;  // 1 / (2 l^2) as a float pair (hi + lo), for the float-pair kernel values
    float vs_f;         // voxel size in FP32
    int cap_leaf, cap_group, search_r, fusion, precision, n_props;
    int emulate;        // Cholesky trailing updates of N > 32 instances on the bf16 tensor cores
    double s2p;         // sigma_prop^2 (surface-property GP, Eq. 6)
    const double* exp_tab;   // 2^(j/256), j = 0..255 (FP64), for exp_neg
    const double* lat_tab;   // exp(-m vs^2 / (2 l^2)), m = 0..kLatticeTable-1 (FP64)
    const float* lat_tab_f;  // the same in FP32
};

constexpr int kLatticeTable = 1024;  // squared integer offsets up to 3 * 15^2 = 675 occur

// e^y for y <= 0 in FP64, table-driven (Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", 1989): y = (256 m + j) ln2/256 + r with
// |r| <= ln2/512, e^y = 2^m * 2^(j/256) * e^r, e^r by its degree-4 Taylor polynomial
// (remainder below 4e-17 relative).  tab[j] = 2^(j/256).  Returns 0 for y < -700.
__device__ __forceinline__ double exp_neg(double y, const double* tab) {
    if (!(y >= -700.0)) return 0.0;
    const double big = 6755399441055744.0;  // 1.5 * 2^52: y * 256/ln2 rounded to an integer
    const double tm = fma(y, 369.3299304675746, big);
    const int ni = __double2loint(tm);
    const double n = tm - big;
    double r = fma(-n, 0x1.62e42fef80000p-9, y);  // ln2/256, high 35 bits (n * hi is exact)
    r = fma(-n, 0x1.1cf79abc9e3b4p-44, r);        // ln2/256, the rest
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    const double s = tab[ni & 255] * p;
    return __longlong_as_double(__double_as_longlong(s) + ((long long)(ni >> 8) << 52));
}

__host__ __device__ inline uint64_t pack_key(int64_t x, int64_t y, int64_t z) {
    return ((uint64_t)(x + kKeyBias) << 42) | ((uint64_t)(y + kKeyBias) << 21) |
           (uint64_t)(z + kKeyBias);
}

__host__ __device__ inline void unpack_key(uint64_t k, int& x, int& y, int& z) {
    x = (int)((int64_t)((k >> 42) & 0x1FFFFF) - kKeyBias);
    y = (int)((int64_t)((k >> 21) & 0x1FFFFF) - kKeyBias);
    z = (int)((int64_t)(k & 0x1FFFFF) - kKeyBias);
}

// floor(v / 8) for negative v too (arithmetic shift)
__host__ __device__ inline int leaf_coord(int v) { return v >> 3; }

// Voxel index ijk = floor(p / vs + 1/2) in IEEE binary64 with explicit round-to-nearest
// operations (no contraction), so every build computes the same integer.
__device__ inline bool voxel_ijk(float px, float py, float pz, double vs, int& i, int& j, int& k) {
    double p[3] = {(double)px, (double)py, (double)pz};
    int o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(p[a])) return false;
        double t = __ddiv_rn(p[a], vs);
        double u = __dadd_rn(t, 0.5);
        double f = floor(u);
        if (!(f > -kIjkLimit && f < kIjkLimit)) return false;
        o[a] = (int)f;
    }
    i = o[0]; j = o[1]; k = o[2];
    return true;
}

// 64-bit finaliser of MurmurHash3 (Appleby), used as the slot hash.
__device__ __forceinline__ uint32_t hash_slot(uint64_t k, uint32_t mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

// Open addressing with linear probing; the probe count is bounded by the capacity.
// Returns the slot, or -1 (and sets kErrTableFull) when the table is full.
__device__ inline int64_t ht_insert(uint64_t* keys, uint32_t mask, uint64_t key, int* err,
                                    bool* inserted = nullptr) {
    uint32_t h = hash_slot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint64_t prev = atomicCAS((unsigned long long*)&keys[h], (unsigned long long)kEmpty,
                                  (unsigned long long)key);
        if (prev == kEmpty) {
            if (inserted) *inserted = true;
            return h;
        }
        if (prev == key) {
            if (inserted) *inserted = false;
            return h;
        }
        h = (h + 1) & mask;
    }
    atomicOr(err, kErrTableFull);
    return -1;
}

__device__ inline int64_t ht_find(const uint64_t* keys, uint32_t mask, uint64_t key) {
    uint32_t h = hash_slot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint64_t k = keys[h];
        if (k == key) return h;
        if (k == kEmpty) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace vgp
