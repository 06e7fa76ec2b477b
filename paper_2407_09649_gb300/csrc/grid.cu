// grid.cu -- sparse leaf grids and instance construction.
//
//   * frame (L-GPDF, Sec. IV-A): voxelise points into a hash of 8^3 leaves with a 512-bit
//     occupancy mask each, one training set per leaf (voxel centres in bit order, capped by
//     stride), the testing voxels (every voxel of each occupied leaf and of its 26
//     neighbours) and the closest-node choice for each testing voxel (Sec. IV-B);
//   * surface (G-GPDF, Sec. IV-D): points binned by leaf;
//   * queries: query leaves, the centre leaf of each one's instance (27-leaf neighbourhood,
//     or a bounded search for the nearest occupied leaf), and instance gathering with the
//     nearest-first cap;
//   * fusion into the global grid (Sec. IV-C, Eqs. 7-9), export and import.
#include <cstdio>

#include "grid.h"

namespace vgp {

namespace {
constexpr int TB = 256;
inline unsigned nblk(int64_t n, int t = TB) { return (unsigned)((n + t - 1) / t); }
}  // namespace

// --------------------------------------------------------------------------------------
// scan (exclusive, int64; out has n + 1 entries)
// --------------------------------------------------------------------------------------
namespace {
constexpr int SCAN_T = 256, SCAN_PER = 4, SCAN_TILE = SCAN_T * SCAN_PER;

__global__ void k_scan_tiles(const int64_t* in, int64_t* out, int64_t n, int64_t* tile_sums) {
    __shared__ int64_t warp_tot[SCAN_T / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t v[SCAN_PER];
    int64_t local = 0;
    for (int k = 0; k < SCAN_PER; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + k;
        v[k] = i < n ? in[i] : 0;
        local += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int64_t woff = 0;
    for (int w = 0; w < wid; ++w) woff += warp_tot[w];
    int64_t run = woff + incl - local;
    for (int k = 0; k < SCAN_PER; ++k) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_PER + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_T - 1) tile_sums[blockIdx.x] = woff + incl;
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* tile_off) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / SCAN_TILE];
}

__global__ void k_set_total(int64_t* out, int64_t n, const int64_t* in) {
    // out[n] = out[n-1] + in[n-1]  (n > 0), 0 otherwise
    out[n] = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

__global__ void k_fill_i64(int64_t* p, int64_t v, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_fill_u64(uint64_t* p, uint64_t v, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_widen_i32(const int32_t* in, int64_t* out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}
__global__ void k_fill_i32(int32_t* p, int32_t v, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
}  // namespace

static void scan_rec(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, Arena& ar, int depth) {
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    Arena::Slot s_sum = (Arena::Slot)(Arena::kScan0 + depth);
    int64_t* sums = (int64_t*)ar.get(s_sum, sizeof(int64_t) * 2 * (tiles + 1), st);
    int64_t* offs = sums + tiles + 1;
    k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, st>>>(in, out, n, sums);
    note_launch();
    if (tiles > 1) {
        if (tiles <= SCAN_TILE) {
            k_scan_tiles<<<1, SCAN_T, 0, st>>>(sums, offs, tiles, sums + tiles);
            note_launch();
        } else {
            scan_rec(sums, offs, tiles, st, ar, depth + 1);
        }
        k_scan_add<<<nblk(n), TB, 0, st>>>(out, n, offs);
        note_launch();
    }
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, Arena& ar) {
    if (n > 0) scan_rec(in, out, n, st, ar, 0);
    k_set_total<<<1, 1, 0, st>>>(out, n, in);
    note_launch();
}

void fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t st) {
    if (n > 0) {
        k_fill_i64<<<nblk(n), TB, 0, st>>>(p, v, n);
        note_launch();
    }
}
void fill_u64(uint64_t* p, uint64_t v, int64_t n, cudaStream_t st) {
    if (n > 0) {
        k_fill_u64<<<nblk(n), TB, 0, st>>>(p, v, n);
        note_launch();
    }
}
void widen_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st) {
    if (n > 0) {
        k_widen_i32<<<nblk(n), TB, 0, st>>>(in, out, n);
        note_launch();
    }
}
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st) {
    if (n > 0) {
        k_fill_i32<<<nblk(n), TB, 0, st>>>(p, v, n);
        note_launch();
    }
}

// --------------------------------------------------------------------------------------
// generic table compaction
// --------------------------------------------------------------------------------------
namespace {
__global__ void k_collect(const uint64_t* keys, int64_t cap, int32_t* slot2idx, int32_t* list,
                          uint64_t* keys_out, int* count, int64_t list_cap, int* err) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= cap) return;
    uint64_t k = keys[s];
    if (k == kEmpty) {
        if (slot2idx) slot2idx[s] = -1;
        return;
    }
    int i = atomicAdd(count, 1);
    if (i >= list_cap) {
        atomicOr(err, kErrCapacity);
        return;
    }
    if (slot2idx) slot2idx[s] = i;
    if (list) list[i] = (int32_t)s;
    if (keys_out) keys_out[i] = k;
}
}  // namespace

void collect_table(const Table& t, int32_t* slot2idx, int32_t* list, uint64_t* keys_out, int* count_dev,
                   int64_t list_cap, int* err, cudaStream_t st) {
    cudaMemsetAsync(count_dev, 0, sizeof(int), st);
    k_collect<<<nblk(t.cap()), TB, 0, st>>>(t.keys, (int64_t)t.cap(), slot2idx, list, keys_out, count_dev,
                                            list_cap, err);
    note_launch();
}

// --------------------------------------------------------------------------------------
// frame (L-GPDF)
// --------------------------------------------------------------------------------------
namespace {
__global__ void k_frame_voxelise(const float* pts, int64_t n, DevParams P, uint64_t* tkeys, uint32_t tmask,
                                 unsigned long long* masks, int* n_valid, int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool valid = false;
    if (i < n) {
        int x, y, z;
        if (voxel_ijk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], P.vs, x, y, z)) {
            uint64_t lk = pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z));
            int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
            int64_t slot = ht_insert(tkeys, tmask, lk, err);
            if (slot >= 0) {
                atomicOr(&masks[slot * 8 + (bit >> 6)], 1ull << (bit & 63));
                valid = true;
            }
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, valid);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_valid, __popc(b));
}

__global__ void k_leaf_counts(const int32_t* list, int nl, const unsigned long long* masks, int cap,
                              int32_t* nocc, int64_t* ninst) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    int s = list[l];
    int c = 0;
    for (int w = 0; w < 8; ++w) c += __popcll(masks[(int64_t)s * 8 + w]);
    nocc[l] = c;
    ninst[l] = c < cap ? c : cap;
}

// One warp per leaf: training voxel centres in bit order with the stride cap.
__global__ void k_leaf_points(const int32_t* list, const uint64_t* lkeys, int nl, const unsigned long long* masks,
                              const int32_t* nocc, const int64_t* inst_off, DevParams P, double* X, double* Xl,
                              float* Xf, char4* Xi, double* centre) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nl) return;
    int s = list[warp];
    unsigned long long wmask = lane < 8 ? masks[(int64_t)s * 8 + lane] : 0ull;
    int wc = __popcll(wmask);
    int pre[9];
    pre[0] = 0;
    for (int w = 0; w < 8; ++w) pre[w + 1] = pre[w] + __shfl_sync(0xffffffffu, wc, w);
    unsigned long long m[8];
    for (int w = 0; w < 8; ++w) m[w] = __shfl_sync(0xffffffffu, wmask, w);
    int lx, ly, lz;
    unpack_key(lkeys[warp], lx, ly, lz);
    double c[3] = {__dmul_rn(__dadd_rn((double)(8 * lx), 3.5), P.vs), __dmul_rn(__dadd_rn((double)(8 * ly), 3.5), P.vs),
                   __dmul_rn(__dadd_rn((double)(8 * lz), 3.5), P.vs)};
    if (lane < 3) centre[3 * (int64_t)warp + lane] = c[lane];
    const int n = nocc[warp];
    const int64_t b0 = inst_off[warp];
    const int N = (int)(inst_off[warp + 1] - b0);
    const int cap = P.cap_leaf;
    for (int k = lane; k < N; k += 32) {
        int rank = n > cap ? (int)(((int64_t)k * n) / cap) : k;
        int w = 0;
        while (rank >= pre[w + 1]) ++w;
        int r = rank - pre[w];
        unsigned lo = (unsigned)(m[w] & 0xffffffffull), hi = (unsigned)(m[w] >> 32);
        int clo = __popc(lo);
        int b = r < clo ? (int)__fns(lo, 0, r + 1) : 32 + (int)__fns(hi, 0, r - clo + 1);
        int bit = w * 64 + b;
        int ijk[3] = {8 * lx + (bit & 7), 8 * ly + ((bit >> 3) & 7), 8 * lz + (bit >> 6)};
        Xi[b0 + k] = make_char4((char)(bit & 7), (char)((bit >> 3) & 7), (char)(bit >> 6), 0);
        for (int a = 0; a < 3; ++a) {
            double g = __dmul_rn((double)ijk[a], P.vs);
            double loc = __dsub_rn(g, c[a]);
            X[3 * (b0 + k) + a] = g;
            Xl[3 * (b0 + k) + a] = loc;
            Xf[3 * (b0 + k) + a] = (float)loc;
        }
    }
}

__global__ void k_dilate(const uint64_t* lkeys, int nl, uint64_t* tkeys, uint32_t tmask, int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)nl * 27) return;
    int l = (int)(i / 27), d = (int)(i % 27);
    int x, y, z;
    unpack_key(lkeys[l], x, y, z);
    ht_insert(tkeys, tmask, pack_key(x + d % 3 - 1, y + (d / 3) % 3 - 1, z + d / 9 - 1), err);
}

// One CTA of 512 threads per testing leaf: closest-node choice for each of its voxels.
// Candidate d enumerates (dz, dy, dx) lexicographically from -1 to 1 (d = 9 dz' + 3 dy' + dx').
__device__ __forceinline__ int choose_node(int t, const int* nb, int mx, int my, int mz) {
    if (nb[13] >= 0) return 13;
    int ijk[3] = {8 * mx + (t & 7), 8 * my + ((t >> 3) & 7), 8 * mz + (t >> 6)};
    int best = -1;
    long long best_d2 = 0;
    for (int d = 0; d < 27; ++d) {
        if (d == 13 || nb[d] < 0) continue;
        int F[3] = {mx + d % 3 - 1, my + (d / 3) % 3 - 1, mz + d / 9 - 1};
        long long d2 = 0;
        for (int a = 0; a < 3; ++a) {
            long long e = 2ll * ijk[a] - (16ll * F[a] + 7);
            d2 += e * e;
        }
        if (best < 0 || d2 < best_d2) {
            best = d;
            best_d2 = d2;
        }
    }
    return best;
}

__global__ void __launch_bounds__(512) k_assign_tests(const uint64_t* tl_keys, const uint64_t* fkeys, uint32_t fmask,
                                                      const int32_t* slot2leaf, int64_t* inst_cnt, int* n_orphan) {
    __shared__ int nb[27];
    __shared__ int cnt[27];
    const int t = threadIdx.x;
    int mx, my, mz;
    unpack_key(tl_keys[blockIdx.x], mx, my, mz);
    if (t < 27) {
        int64_t s = ht_find(fkeys, fmask, pack_key(mx + t % 3 - 1, my + (t / 3) % 3 - 1, mz + t / 9 - 1));
        nb[t] = s >= 0 ? slot2leaf[s] : -1;
        cnt[t] = 0;
    }
    __syncthreads();
    int d = choose_node(t, nb, mx, my, mz);
    if (d >= 0) atomicAdd(&cnt[d], 1);
    else atomicAdd(n_orphan, 1);
    __syncthreads();
    if (t < 27 && cnt[t] > 0) atomicAdd((unsigned long long*)&inst_cnt[nb[t]], (unsigned long long)cnt[t]);
}

__global__ void __launch_bounds__(512) k_scatter_tests(const uint64_t* tl_keys, const uint64_t* fkeys, uint32_t fmask,
                                                       const int32_t* slot2leaf, const int64_t* q_off,
                                                       int64_t* cursor, uint64_t* tkey) {
    __shared__ int nb[27];
    __shared__ int cnt[27];
    __shared__ long long base[27];
    const int t = threadIdx.x;
    int mx, my, mz;
    unpack_key(tl_keys[blockIdx.x], mx, my, mz);
    if (t < 27) {
        int64_t s = ht_find(fkeys, fmask, pack_key(mx + t % 3 - 1, my + (t / 3) % 3 - 1, mz + t / 9 - 1));
        nb[t] = s >= 0 ? slot2leaf[s] : -1;
        cnt[t] = 0;
    }
    __syncthreads();
    int d = choose_node(t, nb, mx, my, mz);
    int r = d >= 0 ? atomicAdd(&cnt[d], 1) : 0;
    __syncthreads();
    if (t < 27 && cnt[t] > 0)
        base[t] = (long long)atomicAdd((unsigned long long*)&cursor[nb[t]], (unsigned long long)cnt[t]);
    __syncthreads();
    if (d < 0) return;
    int I = nb[d];
    int64_t pos = q_off[I] + base[d] + r;
    tkey[pos] = pack_key(8 * mx + (t & 7), 8 * my + ((t >> 3) & 7), 8 * mz + (t >> 6));
}
}  // namespace

void frame_voxelise(const float* pts, int64_t n, const DevParams& P, const Table& t, unsigned long long* masks,
                    int* n_valid, int* err, cudaStream_t st) {
    if (n > 0) {
        k_frame_voxelise<<<nblk(n), TB, 0, st>>>(pts, n, P, t.keys, t.mask, masks, n_valid, err);
        note_launch();
    }
}

void frame_leaf_counts(const int32_t* list, int nl, const unsigned long long* masks, int cap, int32_t* nocc,
                       int64_t* ninst, cudaStream_t st) {
    if (nl > 0) {
        k_leaf_counts<<<nblk(nl), TB, 0, st>>>(list, nl, masks, cap, nocc, ninst);
        note_launch();
    }
}

void frame_leaf_points(const int32_t* list, const uint64_t* lkeys, int nl, const unsigned long long* masks,
                       const int32_t* nocc, const int64_t* inst_off, const DevParams& P, double* X, double* Xl,
                       float* Xf, char4* Xi, double* centre, cudaStream_t st) {
    if (nl > 0) {
        k_leaf_points<<<nblk((int64_t)nl * 32), TB, 0, st>>>(list, lkeys, nl, masks, nocc, inst_off, P, X, Xl, Xf, Xi, centre);
        note_launch();
    }
}

void frame_dilate(const uint64_t* lkeys, int nl, const Table& t, int* err, cudaStream_t st) {
    if (nl > 0) {
        k_dilate<<<nblk((int64_t)nl * 27), TB, 0, st>>>(lkeys, nl, t.keys, t.mask, err);
        note_launch();
    }
}

void frame_assign_tests(const uint64_t* tl_keys, int ntl, const Table& ft, const int32_t* slot2leaf,
                        int64_t* inst_cnt, int* n_orphan, cudaStream_t st) {
    if (ntl > 0) {
        k_assign_tests<<<ntl, 512, 0, st>>>(tl_keys, ft.keys, ft.mask, slot2leaf, inst_cnt, n_orphan);
        note_launch();
    }
}

void frame_scatter_tests(const uint64_t* tl_keys, int ntl, const Table& ft, const int32_t* slot2leaf,
                         const int64_t* q_off, int64_t* cursor, uint64_t* tkey, cudaStream_t st) {
    if (ntl > 0) {
        k_scatter_tests<<<ntl, 512, 0, st>>>(tl_keys, ft.keys, ft.mask, slot2leaf, q_off, cursor, tkey);
        note_launch();
    }
}

// --------------------------------------------------------------------------------------
// ray-cast testing points (Sec. IV-B): surface voxels, voxels along their normals, voxels
// with earlier measurements on the sensor rays; sign by sensor side
// --------------------------------------------------------------------------------------
namespace {
// Warp per frame leaf: every occupied voxel (uncapped), in bit order, at soff[l].
// Surface properties of a frame (Eq. 6): a training point's property is the mean over the
// points in its voxel.  Each point finds its leaf's training index: rank r of its voxel bit in
// the leaf mask; with n > cap occupied voxels the leaf keeps ranks floor(k n / cap), so r is
// kept iff k = ceil(r cap / n) maps back to r.  Sums and counts in FP64 atomics.
__global__ void k_point_props(const float* pts, const float* props, int64_t n, int nc, DevParams P, Table ft,
                              const unsigned long long* masks, const int32_t* slot2leaf, const int32_t* nocc,
                              const int64_t* inst_off, double* ysum, double* ycnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    if (!voxel_ijk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], P.vs, x, y, z)) return;
    const int64_t s = ht_find(ft.keys, ft.mask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)));
    if (s < 0) return;
    const int li = slot2leaf[s];
    if (li < 0) return;
    const int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
    const unsigned long long* mk = masks + s * 8;
    int r = __popcll(mk[bit >> 6] & ((1ull << (bit & 63)) - 1ull));
    for (int w = 0; w < (bit >> 6); ++w) r += __popcll(mk[w]);
    const int no = nocc[li], cap = P.cap_leaf;
    int k = r;
    if (no > cap) {
        k = (int)(((int64_t)r * cap + no - 1) / no);
        if (k >= cap || (int)((int64_t)k * no / cap) != r) return;
    }
    const int64_t t = inst_off[li] + k;
    for (int ch = 0; ch < nc; ++ch) atomicAdd(&ysum[t * nc + ch], (double)props[i * nc + ch]);
    atomicAdd(&ycnt[t], 1.0);
}

__global__ void k_prop_means(double* y, const double* ycnt, int64_t T, int nc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T * nc) return;
    y[i] = y[i] / ycnt[i / nc];
}

__global__ void k_surface_voxels(const int32_t* list, const uint64_t* lkeys, int nl, const unsigned long long* masks,
                                 const int64_t* soff, uint64_t* svox) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nl) return;
    const int s = list[warp];
    int lx, ly, lz;
    unpack_key(lkeys[warp], lx, ly, lz);
    int64_t base = soff[warp];
    for (int w = 0; w < 8; ++w) {
        const unsigned long long m = masks[(int64_t)s * 8 + w];
        for (int half = 0; half < 2; ++half) {
            const unsigned mm = (unsigned)(m >> (32 * half));
            const bool on = (mm >> lane) & 1u;
            const unsigned b = __ballot_sync(0xffffffffu, on);
            if (on) {
                const int bit = w * 64 + half * 32 + lane;
                const int r = __popc(b & ((1u << lane) - 1u));
                svox[base + r] = pack_key(8 * lx + (bit & 7), 8 * ly + ((bit >> 3) & 7), 8 * lz + (bit >> 6));
            }
            base += __popc(b);
        }
    }
}

__device__ __forceinline__ bool frame_occupied(const uint64_t* fkeys, uint32_t fmask, const unsigned long long* masks,
                                               int x, int y, int z) {
    const int64_t s = ht_find(fkeys, fmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)));
    if (s < 0) return false;
    const int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
    return (masks[s * 8 + (bit >> 6)] >> (bit & 63)) & 1ull;
}

__device__ __forceinline__ bool grid_known(const uint64_t* gkeys, uint32_t gmask, const int32_t* slot2pool,
                                           const unsigned long long* known, int x, int y, int z) {
    if (!gkeys) return false;
    const int64_t s = ht_find(gkeys, gmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)));
    if (s < 0) return false;
    const int p = slot2pool[s];
    if (p < 0) return false;
    const int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
    return (known[(int64_t)p * 8 + (bit >> 6)] >> (bit & 63)) & 1ull;
}

__device__ __forceinline__ void add_test(uint64_t* tkeys, uint32_t tmask, unsigned* tflags, int x, int y, int z,
                                         int sign, int* err) {
    if (!(x > -kIjkLimit && x < kIjkLimit && y > -kIjkLimit && y < kIjkLimit && z > -kIjkLimit && z < kIjkLimit)) return;
    const int64_t s = ht_insert(tkeys, tmask, pack_key(x, y, z), err);
    if (s >= 0) atomicOr(&tflags[s], sign > 0 ? 1u : 2u);
}

// Cyclic Jacobi rotations on a symmetric 3x3 (fixed 12 sweeps), every operation explicitly
// rounded so that the result is the same sequence of IEEE operations on every target.
__device__ void jacobi3_rn(double a[3][3], double v[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.0 : 0.0;
    const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 12; ++sweep) {
        for (int r = 0; r < 3; ++r) {
            const int p = PQ[r][0], q = PQ[r][1];
            if (a[p][q] == 0.0) continue;
            const double theta = __ddiv_rn(__dsub_rn(a[q][q], a[p][p]), __dmul_rn(2.0, a[p][q]));
            double t = __ddiv_rn(1.0, __dadd_rn(fabs(theta), __dsqrt_rn(__dadd_rn(__dmul_rn(theta, theta), 1.0))));
            if (theta < 0.0) t = -t;
            const double c = __ddiv_rn(1.0, __dsqrt_rn(__dadd_rn(__dmul_rn(t, t), 1.0)));
            const double sn = __dmul_rn(t, c);
            for (int k = 0; k < 3; ++k) {
                const double akp = a[k][p], akq = a[k][q];
                a[k][p] = __dsub_rn(__dmul_rn(c, akp), __dmul_rn(sn, akq));
                a[k][q] = __dadd_rn(__dmul_rn(sn, akp), __dmul_rn(c, akq));
            }
            for (int k = 0; k < 3; ++k) {
                const double apk = a[p][k], aqk = a[q][k];
                a[p][k] = __dsub_rn(__dmul_rn(c, apk), __dmul_rn(sn, aqk));
                a[q][k] = __dadd_rn(__dmul_rn(sn, apk), __dmul_rn(c, aqk));
            }
            for (int k = 0; k < 3; ++k) {
                const double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = __dsub_rn(__dmul_rn(c, vkp), __dmul_rn(sn, vkq));
                v[k][q] = __dadd_rn(__dmul_rn(sn, vkp), __dmul_rn(c, vkq));
            }
        }
    }
}

// Thread per surface voxel.
__global__ void k_raycast_tests(const uint64_t* svox, int64_t ns, const uint64_t* fkeys, uint32_t fmask,
                                const unsigned long long* fmasks, const uint64_t* gkeys, uint32_t gmask,
                                const int32_t* g_slot2pool, const unsigned long long* g_known, double ox, double oy,
                                double oz, int have_o, int ovx, int ovy, int ovz, double vs, int K, uint64_t* tkeys,
                                uint32_t tmask, unsigned* tflags, int* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ns) return;
    int sv[3];
    unpack_key(svox[i], sv[0], sv[1], sv[2]);
    add_test(tkeys, tmask, tflags, sv[0], sv[1], sv[2], 1, err);
    if (!have_o) return;
    // normal from the exact integer scatter of the occupied 3x3x3 block
    long long cnt = 0, S1[3] = {0, 0, 0}, S2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!frame_occupied(fkeys, fmask, fmasks, sv[0] + dx, sv[1] + dy, sv[2] + dz)) continue;
                const long long o[3] = {dx, dy, dz};
                ++cnt;
                for (int a = 0; a < 3; ++a) {
                    S1[a] += o[a];
                    for (int b = 0; b < 3; ++b) S2[a][b] += o[a] * o[b];
                }
            }
    if (cnt >= 3 && K > 0) {
        double A[3][3], V[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] = (double)(cnt * S2[a][b] - S1[a] * S1[b]);
        jacobi3_rn(A, V);
        int k = 0;
        for (int j = 1; j < 3; ++j)
            if (A[j][j] < A[k][k]) k = j;
        const double nn =
            __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(V[0][k], V[0][k]), __dmul_rn(V[1][k], V[1][k])), __dmul_rn(V[2][k], V[2][k])));
        double nrm[3];
        for (int a = 0; a < 3; ++a) nrm[a] = __ddiv_rn(V[a][k], nn);
        const double org[3] = {ox, oy, oz};
        double e = 0.0;
        for (int a = 0; a < 3; ++a) e = __dadd_rn(e, __dmul_rn(nrm[a], __dsub_rn(org[a], __dmul_rn((double)sv[a], vs))));
        if (e < 0.0)
            for (int a = 0; a < 3; ++a) nrm[a] = -nrm[a];
        for (int kk = -K; kk <= K; ++kk) {
            if (kk == 0) continue;
            int v[3];
            for (int a = 0; a < 3; ++a) v[a] = sv[a] + (int)floor(__dadd_rn(__dmul_rn((double)kk, nrm[a]), 0.5));
            add_test(tkeys, tmask, tflags, v[0], v[1], v[2], kk > 0 ? 1 : -1, err);
        }
    }
    // integer 3D Bresenham from the origin's voxel to the surface voxel (excluded)
    const int a0[3] = {ovx, ovy, ovz};
    long long d[3], st[3], pcur[3] = {a0[0], a0[1], a0[2]};
    for (int k = 0; k < 3; ++k) {
        d[k] = sv[k] > a0[k] ? (long long)sv[k] - a0[k] : (long long)a0[k] - sv[k];
        st[k] = sv[k] > a0[k] ? 1 : -1;
    }
    int m = 0;
    if (d[1] > d[m]) m = 1;
    if (d[2] > d[m]) m = 2;
    const int u = (m + 1) % 3, w = (m + 2) % 3;
    long long eu = 2 * d[u] - d[m], ew = 2 * d[w] - d[m];
    for (long long step = 0; step < d[m]; ++step) {
        if (grid_known(gkeys, gmask, g_slot2pool, g_known, (int)pcur[0], (int)pcur[1], (int)pcur[2]))
            add_test(tkeys, tmask, tflags, (int)pcur[0], (int)pcur[1], (int)pcur[2], 1, err);
        if (eu > 0) {
            pcur[u] += st[u];
            eu -= 2 * d[m];
        }
        if (ew > 0) {
            pcur[w] += st[w];
            ew -= 2 * d[m];
        }
        eu += 2 * d[u];
        ew += 2 * d[w];
        pcur[m] += st[m];
    }
}

// Thread per testing voxel: closest GP leaf (own leaf; else the nearest of the 26 neighbours,
// ties in (dz, dy, dx) order; else the nearest within the search radius, ties to the smaller
// key), or -1.
__global__ void k_assign_list(const uint64_t* tkey, int64_t nt, const uint64_t* fkeys, uint32_t fmask,
                              const int32_t* slot2leaf, int R, int32_t* tinst, int64_t* inst_cnt, int* n_orphan) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int x, y, z;
    unpack_key(tkey[i], x, y, z);
    const int M[3] = {leaf_coord(x), leaf_coord(y), leaf_coord(z)};
    const int ijk[3] = {x, y, z};
    int inst = -1;
    int64_t s = ht_find(fkeys, fmask, pack_key(M[0], M[1], M[2]));
    if (s >= 0) inst = slot2leaf[s];
    if (inst < 0) {
        long long best = 0;
        for (int d = 0; d < 27; ++d) {
            if (d == 13) continue;
            const int F[3] = {M[0] + d % 3 - 1, M[1] + (d / 3) % 3 - 1, M[2] + d / 9 - 1};
            const int64_t fs = ht_find(fkeys, fmask, pack_key(F[0], F[1], F[2]));
            if (fs < 0) continue;
            long long d2 = 0;
            for (int a = 0; a < 3; ++a) {
                const long long e = 2ll * ijk[a] - (16ll * F[a] + 7);
                d2 += e * e;
            }
            if (inst < 0 || d2 < best) {
                best = d2;
                inst = slot2leaf[fs];
            }
        }
    }
    if (inst < 0) {
        long long best = 0;
        uint64_t bkey = 0;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    const int F[3] = {M[0] + dx, M[1] + dy, M[2] + dz};
                    const uint64_t k = pack_key(F[0], F[1], F[2]);
                    const int64_t fs = ht_find(fkeys, fmask, k);
                    if (fs < 0) continue;
                    long long d2 = 0;
                    for (int a = 0; a < 3; ++a) {
                        const long long e = 2ll * ijk[a] - (16ll * F[a] + 7);
                        d2 += e * e;
                    }
                    if (inst < 0 || d2 < best || (d2 == best && k < bkey)) {
                        best = d2;
                        bkey = k;
                        inst = slot2leaf[fs];
                    }
                }
    }
    tinst[i] = inst;
    if (inst >= 0) atomicAdd((unsigned long long*)&inst_cnt[inst], 1ull);
    else atomicAdd(n_orphan, 1);
}

__global__ void k_scatter_list(const uint64_t* tkey, const int8_t* tsign_in, int64_t nt, const int32_t* tinst,
                               const int64_t* q_off, int64_t* cursor, int64_t orphan_base, int* orphan_cursor,
                               uint64_t* gkey, int8_t* gsign) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int I = tinst[i];
    int64_t pos;
    if (I >= 0) pos = q_off[I] + (int64_t)atomicAdd((unsigned long long*)&cursor[I], 1ull);
    else pos = orphan_base + atomicAdd(orphan_cursor, 1);
    gkey[pos] = tkey[i];
    gsign[pos] = tsign_in[i];
}

__global__ void k_collect_tests(const uint64_t* keys, const unsigned* flags, int64_t cap, uint64_t* out_key,
                                int8_t* out_sign, int* count) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= cap || keys[s] == kEmpty) return;
    const int i = atomicAdd(count, 1);
    out_key[i] = keys[s];
    out_sign[i] = (flags[s] & 1u) ? 1 : -1;
}

__global__ void k_orphans_and_sign(int64_t nt, int64_t n_assigned, const int8_t* sign, double* d, double* grad,
                                   double* v, uint8_t* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    if (i >= n_assigned) {
        d[i] = INFINITY;
        v[i] = INFINITY;
        grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = 0.0;
        status[i] = VGP_ST_NO_SUPPORT;
        return;
    }
    if (sign[i] < 0) {
        if (status[i] == VGP_ST_OK || status[i] == VGP_ST_CLAMPED) d[i] = -d[i];
        for (int a = 0; a < 3; ++a) grad[3 * i + a] = -grad[3 * i + a];
    }
}
}  // namespace

void frame_point_props(const float* pts, const float* props, int64_t n, int nc, const DevParams& P, const Table& ft,
                       const unsigned long long* masks, const int32_t* slot2leaf, const int32_t* nocc,
                       const int64_t* inst_off, double* ysum, double* ycnt, cudaStream_t st) {
    if (n <= 0) return;
    k_point_props<<<nblk(n), TB, 0, st>>>(pts, props, n, nc, P, ft, masks, slot2leaf, nocc, inst_off, ysum, ycnt);
    note_launch();
}

void frame_prop_means(double* y, const double* ycnt, int64_t T, int nc, cudaStream_t st) {
    if (T <= 0) return;
    k_prop_means<<<nblk(T * nc), TB, 0, st>>>(y, ycnt, T, nc);
    note_launch();
}

void frame_surface_voxels(const int32_t* list, const uint64_t* lkeys, int nl, const unsigned long long* masks,
                          const int64_t* soff, uint64_t* svox, cudaStream_t st) {
    if (nl > 0) {
        k_surface_voxels<<<nblk((int64_t)nl * 32), TB, 0, st>>>(list, lkeys, nl, masks, soff, svox);
        note_launch();
    }
}

void frame_raycast_tests(const uint64_t* svox, int64_t ns, const Table& ft, const unsigned long long* fmasks,
                         const Table& g, const int32_t* g_slot2pool, const unsigned long long* g_known,
                         const double origin[3], int have_o, const int ov[3], double vs, int K, const Table& tt,
                         unsigned* tflags, int* err, cudaStream_t st) {
    if (ns > 0) {
        k_raycast_tests<<<nblk(ns, 128), 128, 0, st>>>(svox, ns, ft.keys, ft.mask, fmasks, g.keys, g.mask, g_slot2pool,
                                                       g_known, origin[0], origin[1], origin[2], have_o, ov[0], ov[1],
                                                       ov[2], vs, K, tt.keys, tt.mask, tflags, err);
        note_launch();
    }
}

void frame_collect_tests(const Table& tt, const unsigned* tflags, uint64_t* out_key, int8_t* out_sign, int* count,
                         cudaStream_t st) {
    cudaMemsetAsync(count, 0, sizeof(int), st);
    k_collect_tests<<<nblk(tt.cap()), TB, 0, st>>>(tt.keys, tflags, (int64_t)tt.cap(), out_key, out_sign, count);
    note_launch();
}

void frame_assign_list(const uint64_t* tkey, int64_t nt, const Table& ft, const int32_t* slot2leaf, int R,
                       int32_t* tinst, int64_t* inst_cnt, int* n_orphan, cudaStream_t st) {
    if (nt > 0) {
        k_assign_list<<<nblk(nt, 128), 128, 0, st>>>(tkey, nt, ft.keys, ft.mask, slot2leaf, R, tinst, inst_cnt, n_orphan);
        note_launch();
    }
}

void frame_scatter_list(const uint64_t* tkey, const int8_t* tsign, int64_t nt, const int32_t* tinst, const int64_t* q_off,
                        int64_t* cursor, int64_t orphan_base, int* orphan_cursor, uint64_t* gkey, int8_t* gsign,
                        cudaStream_t st) {
    if (nt > 0) {
        k_scatter_list<<<nblk(nt), TB, 0, st>>>(tkey, tsign, nt, tinst, q_off, cursor, orphan_base, orphan_cursor, gkey,
                                               gsign);
        note_launch();
    }
}

void frame_orphans_and_sign(int64_t nt, int64_t n_assigned, const int8_t* sign, double* d, double* grad, double* v,
                            uint8_t* status, cudaStream_t st) {
    if (nt > 0) {
        k_orphans_and_sign<<<nblk(nt), TB, 0, st>>>(nt, n_assigned, sign, d, grad, v, status);
        note_launch();
    }
}

// --------------------------------------------------------------------------------------
// surface (G-GPDF training set)
// --------------------------------------------------------------------------------------
namespace {
__global__ void k_surface_bin(const float* pts, int64_t n, DevParams P, uint64_t* skeys, uint32_t smask,
                              int32_t* pt_slot, int32_t* slot_cnt, int* n_valid, int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool valid = false;
    if (i < n) {
        int x, y, z;
        int32_t s = -1;
        if (voxel_ijk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], P.vs, x, y, z)) {
            int64_t slot = ht_insert(skeys, smask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)), err);
            if (slot >= 0) {
                s = (int32_t)slot;
                atomicAdd(&slot_cnt[slot], 1);
                valid = true;
            }
        }
        pt_slot[i] = s;
    }
    unsigned b = __ballot_sync(0xffffffffu, valid);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_valid, __popc(b));
}

__global__ void k_slot_counts_to_leaf(const int32_t* list, int nl, const int32_t* slot_cnt, int64_t* cnt) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < nl) cnt[l] = slot_cnt[list[l]];
}

__global__ void k_surface_scatter(const int32_t* pt_slot, int64_t n, const int32_t* slot2leaf, const int64_t* off,
                                  int32_t* cursor, int32_t* idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = pt_slot[i];
    if (s < 0) return;
    int l = slot2leaf[s];
    int r = atomicAdd(&cursor[l], 1);
    idx[off[l] + r] = (int32_t)i;
}

// Sort n > 4096 point indices a[0 .. n) ascending in place in global memory, one CTA: a
// bitonic network whose compare-exchanges all put the smaller value first (each merge of size
// k starts by comparing the mirrored positions i and i ^ (k - 1)), so the padding to a power
// of two is virtual: a partner at or beyond n holds +infinity and never moves.
__device__ void sort_long_segment(int32_t* a, int64_t n) {
    int64_t m = 1;
    while (m < n) m <<= 1;
    const int64_t half = m >> 1;
    for (int64_t k = 2; k <= m; k <<= 1) {
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int64_t p = threadIdx.x; p < half; p += blockDim.x) {
                const int64_t i = (p / j) * 2 * j + (p % j);
                const int64_t q = j == (k >> 1) ? i ^ (k - 1) : i + j;
                if (q < n) {
                    const int32_t x = a[i], y = a[q];
                    if (x > y) {
                        a[i] = y;
                        a[q] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Sort each leaf's point indices ascending (bitonic in shared memory up to 4096 points, in
// global memory above), so that the order of every leaf's list, and hence the order of the
// points in every GP instance, does not depend on the order of the scatter's atomics.
__global__ void k_sort_segments(const int64_t* off, int nl, int32_t* idx) {
    __shared__ int32_t buf[4096];
    const int l = blockIdx.x;
    const int64_t b = off[l];
    const int64_t nn = off[l + 1] - b;
    if (nn <= 1) return;
    if (nn > 4096) {
        sort_long_segment(idx + b, nn);
        return;
    }
    const int n = (int)nn;
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) buf[i] = i < n ? idx[b + i] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    bool up = (i & k) == 0;
                    int32_t a = buf[i], c = buf[p];
                    if ((a > c) == up) {
                        buf[i] = c;
                        buf[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) idx[b + i] = buf[i];
}
}  // namespace

void surface_bin(const float* pts, int64_t n, const DevParams& P, const Table& t, int32_t* pt_slot, int32_t* slot_cnt,
                 int* n_valid, int* err, cudaStream_t st) {
    if (n > 0) {
        k_surface_bin<<<nblk(n), TB, 0, st>>>(pts, n, P, t.keys, t.mask, pt_slot, slot_cnt, n_valid, err);
        note_launch();
    }
}

void surface_leaf_counts(const int32_t* list, int nl, const int32_t* slot_cnt, int64_t* cnt, cudaStream_t st) {
    if (nl > 0) {
        k_slot_counts_to_leaf<<<nblk(nl), TB, 0, st>>>(list, nl, slot_cnt, cnt);
        note_launch();
    }
}

void surface_scatter(const int32_t* pt_slot, int64_t n, const int32_t* slot2leaf, const int64_t* off, int32_t* cursor,
                     int32_t* idx, int nl, cudaStream_t st) {
    if (n > 0) {
        k_surface_scatter<<<nblk(n), TB, 0, st>>>(pt_slot, n, slot2leaf, off, cursor, idx);
        note_launch();
    }
    if (nl > 0) {
        k_sort_segments<<<nl, 256, 0, st>>>(off, nl, idx);
        note_launch();
    }
}

// --------------------------------------------------------------------------------------
// queries (G-GPDF)
// --------------------------------------------------------------------------------------
namespace {
__global__ void k_query_leaf(const float* q, int64_t n, DevParams P, uint64_t* qkeys, uint32_t qmask,
                             int32_t* q_slot, int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    int32_t s = -1;
    if (voxel_ijk(q[3 * i], q[3 * i + 1], q[3 * i + 2], P.vs, x, y, z)) {
        int64_t slot = ht_insert(qkeys, qmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)), err);
        s = slot >= 0 ? (int32_t)slot : -2;
    }
    q_slot[i] = s;
}

// Warp per query leaf: centre leaf of its instance.  27-neighbourhood non-empty -> itself;
// else the occupied leaf within Chebyshev radius R with the smallest squared leaf distance,
// ties to the smaller key; none -> kEmpty.
__global__ void k_group_centre(const uint64_t* gkeys, int ng, const uint64_t* skeys, uint32_t smask, int R,
                               uint64_t* gcen) {
    int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (g >= ng) return;
    int mx, my, mz;
    unpack_key(gkeys[g], mx, my, mz);
    bool hit = false;
    if (lane < 27) hit = ht_find(skeys, smask, pack_key(mx + lane % 3 - 1, my + (lane / 3) % 3 - 1, mz + lane / 9 - 1)) >= 0;
    if (__any_sync(0xffffffffu, hit)) {
        if (lane == 0) gcen[g] = gkeys[g];
        return;
    }
    const int side = 2 * R + 1;
    const int total = side * side * side;
    long long bd = 0x7fffffffffffffffll;
    uint64_t bk = kEmpty;
    for (int t = lane; t < total; t += 32) {
        int dx = t % side - R, dy = (t / side) % side - R, dz = t / (side * side) - R;
        uint64_t k = pack_key(mx + dx, my + dy, mz + dz);
        if (ht_find(skeys, smask, k) < 0) continue;
        long long d2 = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
        if (d2 < bd || (d2 == bd && k < bk)) {
            bd = d2;
            bk = k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        long long od = __shfl_xor_sync(0xffffffffu, bd, o);
        unsigned long long ok = __shfl_xor_sync(0xffffffffu, (unsigned long long)bk, o);
        if (od < bd || (od == bd && ok < bk)) {
            bd = od;
            bk = ok;
        }
    }
    if (lane == 0) gcen[g] = bk;
}

__global__ void k_insert_centres(const uint64_t* gcen, int ng, uint64_t* ikeys, uint32_t imask, int* err) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng || gcen[g] == kEmpty) return;
    ht_insert(ikeys, imask, gcen[g], err);
}

// Warp per instance: candidate count over the 27 leaves around the centre.
__global__ void k_inst_count(const uint64_t* ikey, int ni, const uint64_t* skeys, uint32_t smask,
                             const int32_t* sslot2leaf, const int64_t* soff, int cap, int64_t* ncand, int64_t* ninst,
                             int single) {
    int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (I >= ni) return;
    int cx, cy, cz;
    unpack_key(ikey[I], cx, cy, cz);
    int64_t c = 0;
    if (lane < 27 && (!single || lane == 13)) {
        int64_t s = ht_find(skeys, smask, pack_key(cx + lane % 3 - 1, cy + (lane / 3) % 3 - 1, cz + lane / 9 - 1));
        if (s >= 0) {
            int l = sslot2leaf[s];
            c = soff[l + 1] - soff[l];
        }
    }
    c = warp_sum(c);
    if (lane == 0) {
        ncand[I] = c;
        ninst[I] = c < cap ? c : cap;
    }
}

__device__ __forceinline__ uint64_t dist_bits(const float* sp, int32_t i, const double c[3]) {
    double ex = __dsub_rn((double)sp[3 * i], c[0]);
    double ey = __dsub_rn((double)sp[3 * i + 1], c[1]);
    double ez = __dsub_rn((double)sp[3 * i + 2], c[2]);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    return (uint64_t)__double_as_longlong(d2);  // d2 >= 0: the bit pattern orders like the value
}

// Block-wide exclusive prefix of a 0/1 flag (256 threads).
__device__ __forceinline__ int block_excl(int flag, int* warp_tot, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned b = __ballot_sync(0xffffffffu, flag);
    int in_warp = __popc(b & ((1u << lane) - 1));
    if (lane == 0) warp_tot[wid] = __popc(b);
    __syncthreads();
    int off = 0;
    total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        if (w < wid) off += warp_tot[w];
        total += warp_tot[w];
    }
    __syncthreads();
    return off + in_warp;
}

// CTA (256 threads) per instance: gather the 27-leaf candidates; if more than cap, keep the
// cap nearest to the centre-leaf centre (ties by lower point index) by radix selection on
// the FP64 bit pattern, then on the index.  Kept points are written in candidate order.
__global__ void __launch_bounds__(256) k_inst_gather(const uint64_t* ikey, const uint64_t* skeys, uint32_t smask,
                                                     const int32_t* sslot2leaf, const int64_t* soff, const int32_t* sidx,
                                                     const float* spts, const int64_t* ncand, const int64_t* inst_off,
                                                     DevParams P, double* Xl, float* Xf, int64_t* gidx, double* centre,
                                                     int single) {
    __shared__ int64_t lo[27], cnt[28];
    __shared__ unsigned hist[256];
    __shared__ int warp_tot[8];
    __shared__ uint64_t s_prefix;
    __shared__ int s_need;
    __shared__ int s_rem_ties;
    __shared__ int64_t s_pos;
    const int I = blockIdx.x, t = threadIdx.x;
    int cx, cy, cz;
    unpack_key(ikey[I], cx, cy, cz);
    const double c[3] = {__dmul_rn(__dadd_rn((double)(8 * cx), 3.5), P.vs), __dmul_rn(__dadd_rn((double)(8 * cy), 3.5), P.vs),
                         __dmul_rn(__dadd_rn((double)(8 * cz), 3.5), P.vs)};
    if (t < 3) centre[3 * (int64_t)I + t] = c[t];
    if (t < 27) {
        int64_t s = (single && t != 13) ? -1
                                        : ht_find(skeys, smask, pack_key(cx + t % 3 - 1, cy + (t / 3) % 3 - 1, cz + t / 9 - 1));
        if (s >= 0) {
            int l = sslot2leaf[s];
            lo[t] = soff[l];
            cnt[t + 1] = soff[l + 1] - soff[l];
        } else {
            lo[t] = 0;
            cnt[t + 1] = 0;
        }
    }
    __syncthreads();
    if (t == 0) {
        cnt[0] = 0;
        for (int k = 0; k < 27; ++k) cnt[k + 1] += cnt[k];
    }
    __syncthreads();
    const int64_t nc = cnt[27];
    const int64_t b0 = inst_off[I];
    const int N = (int)(inst_off[I + 1] - b0);
    auto cand = [&](int64_t r) -> int32_t {
        int k = 0;
        while (r >= cnt[k + 1]) ++k;
        return sidx[lo[k] + (r - cnt[k])];
    };
    auto emit = [&](int64_t pos, int32_t i) {
        for (int a = 0; a < 3; ++a) {
            double v = __dsub_rn((double)spts[3 * i + a], c[a]);
            Xl[3 * (b0 + pos) + a] = v;
            Xf[3 * (b0 + pos) + a] = (float)v;
        }
        gidx[b0 + pos] = i;
    };
    if (nc <= N) {
        for (int64_t r = t; r < nc; r += blockDim.x) emit(r, cand(r));
        return;
    }
    // radix select the N-th smallest distance (MSB first, 8 bits per pass)
    if (t == 0) {
        s_prefix = 0;
        s_need = N;
    }
    __syncthreads();
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        hist[t] = 0;
        __syncthreads();
        const uint64_t pmask = pass == 0 ? 0ull : (~0ull << (shift + 8));
        for (int64_t r = t; r < nc; r += blockDim.x) {
            uint64_t k = dist_bits(spts, cand(r), c);
            if ((k & pmask) == (s_prefix & pmask)) atomicAdd(&hist[(k >> shift) & 255], 1u);
        }
        __syncthreads();
        if (t == 0) {
            int need = s_need;
            int acc = 0, bsel = 255;
            for (int b = 0; b < 256; ++b) {
                if (acc + (int)hist[b] >= need) {
                    bsel = b;
                    break;
                }
                acc += hist[b];
            }
            s_need = need - acc;
            s_prefix |= (uint64_t)bsel << shift;
        }
        __syncthreads();
    }
    const uint64_t thr = s_prefix;  // N-th smallest distance bits; s_need of its ties are kept
    // among ties, keep the s_need smallest indices: radix select on the index (31 bits)
    if (t == 0) s_rem_ties = s_need;
    __syncthreads();
    uint32_t iprefix = 0;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        hist[t] = 0;
        __syncthreads();
        const uint32_t pmask = pass == 0 ? 0u : (~0u << (shift + 8));
        for (int64_t r = t; r < nc; r += blockDim.x) {
            int32_t i = cand(r);
            if (dist_bits(spts, i, c) != thr) continue;
            if (((uint32_t)i & pmask) == (iprefix & pmask)) atomicAdd(&hist[((uint32_t)i >> shift) & 255], 1u);
        }
        __syncthreads();
        if (t == 0) {
            int acc = 0, bsel = 255;
            for (int b = 0; b < 256; ++b) {
                if (acc + (int)hist[b] >= s_rem_ties) {
                    bsel = b;
                    break;
                }
                acc += hist[b];
            }
            s_rem_ties -= acc;
            hist[0] = bsel;  // broadcast through shared memory
        }
        __syncthreads();
        iprefix |= (uint32_t)hist[0] << shift;
        __syncthreads();
    }
    const uint32_t ithr = iprefix;  // keep ties with index <= ithr
    // write kept candidates in candidate order (block-wide prefix of the keep flag)
    if (t == 0) s_pos = 0;
    __syncthreads();
    for (int64_t r0 = 0; r0 < nc; r0 += blockDim.x) {
        int64_t r = r0 + t;
        int32_t i = 0;
        int keep = 0;
        if (r < nc) {
            i = cand(r);
            uint64_t k = dist_bits(spts, i, c);
            keep = k < thr || (k == thr && (uint32_t)i <= ithr);
        }
        int total;
        int off = block_excl(keep, warp_tot, total);
        if (keep && s_pos + off < N) emit(s_pos + off, i);
        __syncthreads();
        if (t == 0) s_pos += total;
        __syncthreads();
    }
}

__global__ void k_query_route(const int32_t* q_slot, int64_t n, const int32_t* slot2group, const uint64_t* gcen,
                              const uint64_t* ikeys, uint32_t imask, const int32_t* islot2inst, int32_t* q_inst,
                              int64_t* inst_qcnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = q_slot[i];
    int32_t I = -3;  // bad input
    if (s >= 0) {
        uint64_t ck = gcen[slot2group[s]];
        if (ck == kEmpty) {
            I = -1;  // no support
        } else {
            int64_t is = ht_find(ikeys, imask, ck);
            I = is >= 0 ? islot2inst[is] : -1;
        }
    } else if (s == -2) {
        I = -2;  // table full (reported through err)
    }
    q_inst[i] = I;
    if (I >= 0) atomicAdd((unsigned long long*)&inst_qcnt[I], 1ull);
}

__global__ void k_query_scatter(const int32_t* q_inst, int64_t n, const int64_t* q_off, int64_t* cursor, int64_t* qidx,
                                double* d, double* grad, double* var, uint8_t* status) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t I = q_inst[i];
    if (I >= 0) {
        int64_t r = (int64_t)atomicAdd((unsigned long long*)&cursor[I], 1ull);
        qidx[q_off[I] + r] = i;
        return;
    }
    d[i] = INFINITY;
    if (grad) grad[3 * i] = grad[3 * i + 1] = grad[3 * i + 2] = 0.0;
    if (var) var[i] = INFINITY;
    if (status) status[i] = I == -1 ? VGP_ST_NO_SUPPORT : VGP_ST_BAD_INPUT;
}
}  // namespace

void query_leaf(const float* q, int64_t n, const DevParams& P, const Table& t, int32_t* q_slot, int* err, cudaStream_t st) {
    if (n > 0) {
        k_query_leaf<<<nblk(n), TB, 0, st>>>(q, n, P, t.keys, t.mask, q_slot, err);
        note_launch();
    }
}

void group_centre(const uint64_t* gkeys, int ng, const Table& s, int R, uint64_t* gcen, cudaStream_t st) {
    if (ng > 0) {
        k_group_centre<<<nblk((int64_t)ng * 32), TB, 0, st>>>(gkeys, ng, s.keys, s.mask, R, gcen);
        note_launch();
    }
}

void insert_centres(const uint64_t* gcen, int ng, const Table& it, int* err, cudaStream_t st) {
    if (ng > 0) {
        k_insert_centres<<<nblk(ng), TB, 0, st>>>(gcen, ng, it.keys, it.mask, err);
        note_launch();
    }
}

void inst_count(const uint64_t* ikey, int ni, const Table& s, const int32_t* sslot2leaf, const int64_t* soff, int cap,
                int64_t* ncand, int64_t* ninst, cudaStream_t st, int single) {
    if (ni > 0) {
        k_inst_count<<<nblk((int64_t)ni * 32), TB, 0, st>>>(ikey, ni, s.keys, s.mask, sslot2leaf, soff, cap, ncand, ninst, single);
        note_launch();
    }
}

void inst_gather(const uint64_t* ikey, int ni, const Table& s, const int32_t* sslot2leaf, const int64_t* soff,
                 const int32_t* sidx, const float* spts, const int64_t* ncand, const int64_t* inst_off,
                 const DevParams& P, double* Xl, float* Xf, int64_t* gidx, double* centre, cudaStream_t st, int single) {
    if (ni > 0)
        k_inst_gather<<<ni, 256, 0, st>>>(ikey, s.keys, s.mask, sslot2leaf, soff, sidx, spts, ncand, inst_off, P, Xl, Xf,
                                          gidx, centre, single);
        note_launch();
}

void query_route(const int32_t* q_slot, int64_t n, const int32_t* slot2group, const uint64_t* gcen, const Table& it,
                 const int32_t* islot2inst, int32_t* q_inst, int64_t* inst_qcnt, cudaStream_t st) {
    if (n > 0)
        k_query_route<<<nblk(n), TB, 0, st>>>(q_slot, n, slot2group, gcen, it.keys, it.mask, islot2inst, q_inst, inst_qcnt);
        note_launch();
}

void query_scatter(const int32_t* q_inst, int64_t n, const int64_t* q_off, int64_t* cursor, int64_t* qidx, double* d,
                   double* grad, double* var, uint8_t* status, cudaStream_t st) {
    if (n > 0) {
        k_query_scatter<<<nblk(n), TB, 0, st>>>(q_inst, n, q_off, cursor, qidx, d, grad, var, status);
        note_launch();
    }
}

// --------------------------------------------------------------------------------------
// G-GPDF as per-leaf GPs blended by a smooth minimum (Sec. IV-D, Eq. 10)
// --------------------------------------------------------------------------------------
namespace {
// Warp per query group: every occupied leaf of the centre leaf's 27-neighbourhood is a node.
__global__ void k_smooth_nodes(const uint64_t* gcen, int ng, const uint64_t* skeys, uint32_t smask, uint64_t* ikeys,
                               uint32_t imask, int* err) {
    int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (g >= ng || lane >= 27 || gcen[g] == kEmpty) return;
    int cx, cy, cz;
    unpack_key(gcen[g], cx, cy, cz);
    const uint64_t k = pack_key(cx + lane % 3 - 1, cy + (lane / 3) % 3 - 1, cz + lane / 9 - 1);
    if (ht_find(skeys, smask, k) >= 0) ht_insert(ikeys, imask, k, err);
}

// Thread per query: the Q nodes nearest to the query point (FP64 squared distance to the leaf
// centre, ties to the smaller key) among the occupied leaves around its centre leaf; one
// (query, node) pair per chosen node, pair id = query * Q + rank.
__global__ void k_smooth_pairs(const float* q, int64_t n, const int32_t* q_slot, const int32_t* slot2group,
                               const uint64_t* gcen, const uint64_t* skeys, uint32_t smask, const uint64_t* ikeys,
                               uint32_t imask, const int32_t* islot2inst, DevParams P, int Q, int32_t* pair_inst,
                               uint8_t* n_nodes, int64_t* inst_cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int t = 0; t < Q; ++t) pair_inst[i * Q + t] = -1;
    n_nodes[i] = 0;
    const int32_t s = q_slot[i];
    if (s < 0) return;
    const uint64_t ck = gcen[slot2group[s]];
    if (ck == kEmpty) return;
    int cx, cy, cz;
    unpack_key(ck, cx, cy, cz);
    const double xs[3] = {(double)q[3 * i], (double)q[3 * i + 1], (double)q[3 * i + 2]};
    double bd[27];
    uint64_t bk[27];
    int nn = 0;
    for (int t = 0; t < 27; ++t) {
        const int F[3] = {cx + t % 3 - 1, cy + (t / 3) % 3 - 1, cz + t / 9 - 1};
        const uint64_t k = pack_key(F[0], F[1], F[2]);
        if (ht_find(skeys, smask, k) < 0) continue;
        double e2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double c = __dmul_rn(__dadd_rn((double)(8 * F[a]), 3.5), P.vs);
            const double e = __dsub_rn(xs[a], c);
            e2 = __dadd_rn(e2, __dmul_rn(e, e));
        }
        int pos = nn++;
        while (pos > 0 && (bd[pos - 1] > e2 || (bd[pos - 1] == e2 && bk[pos - 1] > k))) {
            bd[pos] = bd[pos - 1];
            bk[pos] = bk[pos - 1];
            --pos;
        }
        bd[pos] = e2;
        bk[pos] = k;
    }
    const int use = nn < Q ? nn : Q;
    for (int t = 0; t < use; ++t) {
        const int64_t is = ht_find(ikeys, imask, bk[t]);
        const int I = is >= 0 ? islot2inst[is] : -1;
        pair_inst[i * Q + t] = I;
        if (I >= 0) atomicAdd((unsigned long long*)&inst_cnt[I], 1ull);
    }
    n_nodes[i] = (uint8_t)use;
}

__global__ void k_smooth_scatter(const int32_t* pair_inst, int64_t npairs, const int64_t* q_off, int64_t* cursor,
                                 int64_t* qidx) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int32_t I = pair_inst[p];
    if (I < 0) return;
    const int64_t r = (int64_t)atomicAdd((unsigned long long*)&cursor[I], 1ull);
    qidx[q_off[I] + r] = p;
}

// Thread per query: d = sum_q w_q d_q / sum_q w_q, w_q = exp(-lambda (d_q - min d)) over the
// valid nodes; gradient = plain average of their gradients; variance = weighted average.
__global__ void k_smooth_blend(int64_t n, int Q, const int32_t* q_slot, const uint8_t* n_nodes, const double* pd,
                               const double* pg, const double* pv, const uint8_t* ps, double lambda, DevParams P,
                               double* d, double* grad, double* var, uint8_t* status) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nn = n_nodes[i];
    double dd, g[3] = {0.0, 0.0, 0.0}, vv = INFINITY;
    int st;
    if (q_slot[i] < 0 || nn == 0) {
        st = q_slot[i] < 0 ? VGP_ST_BAD_INPUT : VGP_ST_NO_SUPPORT;
        dd = INFINITY;
    } else {
        double dmin = INFINITY;
        int n_ok = 0;
        for (int t = 0; t < nn; ++t)
            if (ps[i * Q + t] == VGP_ST_OK) {
                ++n_ok;
                dmin = fmin(dmin, pd[i * Q + t]);
            }
        if (n_ok == 0) {
            st = ps[i * Q];
            dd = st == VGP_ST_CLAMPED ? P.d_max : INFINITY;
        } else {
            double sw = 0.0, swd = 0.0, swv = 0.0;
            for (int t = 0; t < nn; ++t) {
                const int64_t p = i * Q + t;
                if (ps[p] != VGP_ST_OK) continue;
                const double w = exp(-lambda * (pd[p] - dmin));
                sw += w;
                swd += w * pd[p];
                if (pv) swv += w * pv[p];
                for (int a = 0; a < 3; ++a) g[a] += pg[3 * p + a];
            }
            dd = swd / sw;
            vv = pv ? swv / sw : NAN;
            for (int a = 0; a < 3; ++a) g[a] /= (double)n_ok;
            st = VGP_ST_OK;
        }
    }
    d[i] = dd;
    if (grad)
        for (int a = 0; a < 3; ++a) grad[3 * i + a] = g[a];
    if (var) var[i] = vv;
    if (status) status[i] = (uint8_t)st;
}
}  // namespace

void smooth_nodes(const uint64_t* gcen, int ng, const Table& s, const Table& it, int* err, cudaStream_t st) {
    if (ng > 0) {
        k_smooth_nodes<<<nblk((int64_t)ng * 32), TB, 0, st>>>(gcen, ng, s.keys, s.mask, it.keys, it.mask, err);
        note_launch();
    }
}

void smooth_pairs(const float* q, int64_t n, const int32_t* q_slot, const int32_t* slot2group, const uint64_t* gcen,
                  const Table& s, const Table& it, const int32_t* islot2inst, const DevParams& P, int Q,
                  int32_t* pair_inst, uint8_t* n_nodes, int64_t* inst_cnt, cudaStream_t st) {
    if (n > 0) {
        k_smooth_pairs<<<nblk(n, 128), 128, 0, st>>>(q, n, q_slot, slot2group, gcen, s.keys, s.mask, it.keys, it.mask,
                                                     islot2inst, P, Q, pair_inst, n_nodes, inst_cnt);
        note_launch();
    }
}

void smooth_scatter(const int32_t* pair_inst, int64_t npairs, const int64_t* q_off, int64_t* cursor, int64_t* qidx,
                    cudaStream_t st) {
    if (npairs > 0) {
        k_smooth_scatter<<<nblk(npairs), TB, 0, st>>>(pair_inst, npairs, q_off, cursor, qidx);
        note_launch();
    }
}

void smooth_blend(int64_t n, int Q, const int32_t* q_slot, const uint8_t* n_nodes, const double* pd, const double* pg,
                  const double* pv, const uint8_t* ps, double lambda, const DevParams& P, double* d, double* grad,
                  double* var, uint8_t* status, cudaStream_t st) {
    if (n > 0) {
        k_smooth_blend<<<nblk(n), TB, 0, st>>>(n, Q, q_slot, n_nodes, pd, pg, pv, ps, lambda, P, d, grad, var, status);
        note_launch();
    }
}

// --------------------------------------------------------------------------------------
// fusion (Eqs. 7-9) into the global grid
// --------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ bool fusable(int mode, uint8_t st, double d, double v) {
    if (st != VGP_ST_OK || !isfinite(d) || !isfinite(v) || !(v > 0.0)) return false;
    return mode == 0 || v < 1.0;
}

__global__ void k_fuse_clear(int32_t* flags, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] &= ~1;
}

__global__ void k_fuse_insert(const uint64_t* vkey, const double* d, const double* v, const uint8_t* st, int64_t n,
                              int mode, uint64_t* gkeys, uint32_t gmask, int32_t* slot2pool, int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !fusable(mode, st[i], d[i], v[i])) return;
    int x, y, z;
    unpack_key(vkey[i], x, y, z);
    bool ins = false;
    int64_t s = ht_insert(gkeys, gmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)), err, &ins);
    if (s >= 0 && ins) slot2pool[s] = -2;
}

__global__ void k_fuse_alloc(int32_t* slot2pool, int64_t cap, int* pool_count, int pool_cap,
                             unsigned long long* known, int32_t* flags, int* err, PropGrid pg) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= cap || slot2pool[s] != -2) return;
    int p = atomicAdd(pool_count, 1);
    if (p >= pool_cap) {
        atomicOr(err, kErrCapacity);
        slot2pool[s] = -1;
        return;
    }
    slot2pool[s] = p;
    for (int w = 0; w < 8; ++w) known[(int64_t)p * 8 + w] = 0ull;
    flags[p] = 0;
    if (pg.nc > 0)
        for (int e = 0; e < 512; ++e) {
            pg.W[(int64_t)p * 512 + e] = __longlong_as_double(0x7ff8000000000000ll);
            for (int ch = 0; ch < pg.nc; ++ch) pg.C[((int64_t)p * 512 + e) * pg.nc + ch] = __longlong_as_double(0x7ff8000000000000ll);
        }
}

// Surface-property fusion: the rules of the distance fusion (Eqs. 8-9) applied to every
// channel with the shared variance (weight) W; W = NaN takes the first estimate.
__device__ __forceinline__ void fuse_props(int mode, double* C, double* W, const double* c, double w, int nc) {
    if (isnan(*W)) {
        for (int ch = 0; ch < nc; ++ch) C[ch] = c[ch];
        *W = mode == 0 ? w : 1.0 - w;
        return;
    }
    if (mode == 0) {
        const double Wp = *W;
        const double a = Wp / (Wp + w), b = w / (Wp + w);
        for (int ch = 0; ch < nc; ++ch) C[ch] = a * c[ch] + b * C[ch];
        *W = 1.0 / (1.0 / Wp + 1.0 / w);
    } else {
        const double Wp = *W, ww = 1.0 - w;
        const double a = ww / (Wp + ww), b = Wp / (Wp + ww);
        for (int ch = 0; ch < nc; ++ch) C[ch] = a * c[ch] + b * C[ch];
        *W = Wp + ww;
    }
}

__global__ void k_fuse_update(const uint64_t* vkey, const double* d, const double* v, const uint8_t* st, int64_t n,
                              int mode, const uint64_t* gkeys, uint32_t gmask, const int32_t* slot2pool,
                              unsigned long long* known, double* D, double* V, int32_t* flags, PropIn pin,
                              PropGrid pg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !fusable(mode, st[i], d[i], v[i])) return;
    int x, y, z;
    unpack_key(vkey[i], x, y, z);
    int64_t s = ht_find(gkeys, gmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)));
    if (s < 0) return;
    int p = slot2pool[s];
    if (p < 0) return;
    int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
    int64_t e = (int64_t)p * 512 + bit;
    unsigned long long m = 1ull << (bit & 63);
    unsigned long long old = atomicOr(&known[(int64_t)p * 8 + (bit >> 6)], m);
    const double dn = d[i], vn = v[i];
    if (!(old & m)) {
        D[e] = dn;
        V[e] = mode == 0 ? vn : 1.0 - vn;
    } else if (mode == 0) {
        const double Vp = V[e];
        const double a = Vp / (Vp + vn), b = vn / (Vp + vn);
        D[e] = a * dn + b * D[e];
        V[e] = 1.0 / (1.0 / Vp + 1.0 / vn);
    } else {
        const double Vp = V[e], w = 1.0 - vn;
        const double a = w / (Vp + w), b = Vp / (Vp + w);
        D[e] = a * dn + b * D[e];
        V[e] = Vp + w;
    }
    atomicOr(&flags[p], 3);
    if (pg.nc > 0 && pin.c) {
        // properties fuse where the distance fuses and their estimate is valid
        const int nc = pg.nc;
        const double wn = pin.w[i];
        bool okp = isfinite(wn) && wn > 0.0 && (mode == 0 || wn < 1.0);
        double cv[4];
        for (int ch = 0; ch < nc; ++ch) {
            cv[ch] = pin.c[i * nc + ch];
            okp = okp && isfinite(cv[ch]);
        }
        if (okp) fuse_props(mode, pg.C + e * nc, pg.W + e, cv, wn, nc);
    }
}

__global__ void k_export_props(const uint64_t* gkeys, int64_t cap, const int32_t* slot2pool,
                               const unsigned long long* known, PropGrid pg, int* count, uint64_t* okey, double* oC,
                               double* oW) {
    int64_t s = blockIdx.x;
    if (s >= cap || gkeys[s] == kEmpty) return;
    int p = slot2pool[s];
    if (p < 0) return;
    int bit = threadIdx.x;
    if (!((known[(int64_t)p * 8 + (bit >> 6)] >> (bit & 63)) & 1ull)) return;
    int lx, ly, lz;
    unpack_key(gkeys[s], lx, ly, lz);
    int o = atomicAdd(count, 1);
    okey[o] = pack_key(8 * lx + (bit & 7), 8 * ly + ((bit >> 3) & 7), 8 * lz + (bit >> 6));
    const int64_t e = (int64_t)p * 512 + bit;
    for (int ch = 0; ch < pg.nc; ++ch) oC[(int64_t)o * pg.nc + ch] = pg.C[e * pg.nc + ch];
    oW[o] = pg.W[e];
}

__global__ void k_import_props(const uint64_t* vkey, const double* iC, const double* iW, int64_t n,
                               const uint64_t* gkeys, uint32_t gmask, const int32_t* slot2pool,
                               const unsigned long long* known, PropGrid pg) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    unpack_key(vkey[i], x, y, z);
    int64_t s = ht_find(gkeys, gmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)));
    if (s < 0) return;
    int p = slot2pool[s];
    if (p < 0) return;
    int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
    if (!((known[(int64_t)p * 8 + (bit >> 6)] >> (bit & 63)) & 1ull)) return;
    const int64_t e = (int64_t)p * 512 + bit;
    for (int ch = 0; ch < pg.nc; ++ch) pg.C[e * pg.nc + ch] = iC[i * pg.nc + ch];
    pg.W[e] = iW[i];
}

__global__ void k_export(const uint64_t* gkeys, int64_t cap, const int32_t* slot2pool, const unsigned long long* known,
                         const double* D, const double* V, const int32_t* flags, int* count, uint64_t* okey, double* oD,
                         double* oV, uint8_t* ofl) {
    // one CTA of 512 threads per table slot range: thread = voxel bit of slot blockIdx.x
    int64_t s = blockIdx.x;
    if (s >= cap || gkeys[s] == kEmpty) return;
    int p = slot2pool[s];
    if (p < 0) return;
    int bit = threadIdx.x;
    if (!((known[(int64_t)p * 8 + (bit >> 6)] >> (bit & 63)) & 1ull)) return;
    int lx, ly, lz;
    unpack_key(gkeys[s], lx, ly, lz);
    int o = atomicAdd(count, 1);
    okey[o] = pack_key(8 * lx + (bit & 7), 8 * ly + ((bit >> 3) & 7), 8 * lz + (bit >> 6));
    oD[o] = D[(int64_t)p * 512 + bit];
    oV[o] = V[(int64_t)p * 512 + bit];
    ofl[o] = (uint8_t)flags[p];
}

__global__ void k_import_insert(const uint64_t* vkey, int64_t n, uint64_t* gkeys, uint32_t gmask, int32_t* slot2pool,
                                int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    unpack_key(vkey[i], x, y, z);
    bool ins = false;
    int64_t s = ht_insert(gkeys, gmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)), err, &ins);
    if (s >= 0 && ins) slot2pool[s] = -2;
}

__global__ void k_import_set(const uint64_t* vkey, const double* iD, const double* iV, const uint8_t* ifl, int64_t n,
                             const uint64_t* gkeys, uint32_t gmask, const int32_t* slot2pool, unsigned long long* known,
                             double* D, double* V, int32_t* flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    unpack_key(vkey[i], x, y, z);
    int64_t s = ht_find(gkeys, gmask, pack_key(leaf_coord(x), leaf_coord(y), leaf_coord(z)));
    if (s < 0) return;
    int p = slot2pool[s];
    if (p < 0) return;
    int bit = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
    atomicOr(&known[(int64_t)p * 8 + (bit >> 6)], 1ull << (bit & 63));
    D[(int64_t)p * 512 + bit] = iD[i];
    V[(int64_t)p * 512 + bit] = iV[i];
    atomicOr(&flags[p], (int)ifl[i]);
}

__global__ void k_rehash(const uint64_t* okeys, const int32_t* oslot2pool, int64_t ocap, uint64_t* nkeys, uint32_t nmask,
                         int32_t* nslot2pool, int* err) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= ocap || okeys[s] == kEmpty) return;
    int64_t t = ht_insert(nkeys, nmask, okeys[s], err);
    if (t >= 0) nslot2pool[t] = oslot2pool[s];
}
}  // namespace

void fuse_clear_flags(int32_t* flags, int n, cudaStream_t st) {
    if (n > 0) {
        k_fuse_clear<<<nblk(n), TB, 0, st>>>(flags, n);
        note_launch();
    }
}

void fuse_insert(const uint64_t* vkey, const double* d, const double* v, const uint8_t* s, int64_t n, int mode,
                 const Table& g, int32_t* slot2pool, int* err, cudaStream_t st) {
    if (n > 0) {
        k_fuse_insert<<<nblk(n), TB, 0, st>>>(vkey, d, v, s, n, mode, g.keys, g.mask, slot2pool, err);
        note_launch();
    }
}

void fuse_alloc(int32_t* slot2pool, const Table& g, int* pool_count, int pool_cap, unsigned long long* known,
                int32_t* flags, int* err, const PropGrid& pg, cudaStream_t st) {
    k_fuse_alloc<<<nblk(g.cap()), TB, 0, st>>>(slot2pool, (int64_t)g.cap(), pool_count, pool_cap, known, flags, err,
                                               pg);
    note_launch();
}

void fuse_update(const uint64_t* vkey, const double* d, const double* v, const uint8_t* s, int64_t n, int mode,
                 const Table& g, const int32_t* slot2pool, unsigned long long* known, double* D, double* V,
                 int32_t* flags, const PropIn& pin, const PropGrid& pg, cudaStream_t st) {
    if (n > 0) {
        k_fuse_update<<<nblk(n), TB, 0, st>>>(vkey, d, v, s, n, mode, g.keys, g.mask, slot2pool, known, D, V, flags,
                                              pin, pg);
        note_launch();
    }
}

void grid_export_props(const Table& g, const int32_t* slot2pool, const unsigned long long* known, const PropGrid& pg,
                       int* count, uint64_t* okey, double* oC, double* oW, cudaStream_t st) {
    cudaMemsetAsync(count, 0, sizeof(int), st);
    k_export_props<<<(unsigned)g.cap(), 512, 0, st>>>(g.keys, (int64_t)g.cap(), slot2pool, known, pg, count, okey, oC,
                                                      oW);
    note_launch();
}

void grid_import_props(const uint64_t* vkey, const double* iC, const double* iW, int64_t n, const Table& g,
                       const int32_t* slot2pool, const unsigned long long* known, const PropGrid& pg, cudaStream_t st) {
    if (n <= 0 || pg.nc <= 0) return;
    k_import_props<<<nblk(n), TB, 0, st>>>(vkey, iC, iW, n, g.keys, g.mask, slot2pool, known, pg);
    note_launch();
}

void grid_export(const Table& g, const int32_t* slot2pool, const unsigned long long* known, const double* D,
                 const double* V, const int32_t* flags, int* count, uint64_t* okey, double* oD, double* oV,
                 uint8_t* ofl, cudaStream_t st) {
    cudaMemsetAsync(count, 0, sizeof(int), st);
    k_export<<<(unsigned)g.cap(), 512, 0, st>>>(g.keys, (int64_t)g.cap(), slot2pool, known, D, V, flags, count, okey, oD,
                                                  oV, ofl);
    note_launch();
}

void grid_import(const uint64_t* vkey, const double* iD, const double* iV, const uint8_t* ifl, int64_t n, const Table& g,
                 int32_t* slot2pool, int* pool_count, int pool_cap, unsigned long long* known, double* D, double* V,
                 int32_t* flags, int* err, const PropGrid& pg, cudaStream_t st) {
    if (n <= 0) return;
    k_import_insert<<<nblk(n), TB, 0, st>>>(vkey, n, g.keys, g.mask, slot2pool, err);
    note_launch();
    fuse_alloc(slot2pool, g, pool_count, pool_cap, known, flags, err, pg, st);
    k_import_set<<<nblk(n), TB, 0, st>>>(vkey, iD, iV, ifl, n, g.keys, g.mask, slot2pool, known, D, V, flags);
    note_launch();
}

void grid_rehash(const Table& o, const int32_t* oslot2pool, const Table& nt, int32_t* nslot2pool, int* err,
                 cudaStream_t st) {
    k_rehash<<<nblk(o.cap()), TB, 0, st>>>(o.keys, oslot2pool, (int64_t)o.cap(), nt.keys, nt.mask, nslot2pool, err);
    note_launch();
}

}  // namespace vgp
