// mesh.cu -- zero crossings and marching cubes over the fused global grid (Sec. IV-D).
//
// The fused distance D of a voxel sits at its centre ijk * vs; a voxel is inside when D < 0.
// A zero crossing lies on every axis edge between two known neighbouring voxels whose insides
// differ, at p_axis = (a_axis + t) vs with t = D_a / (D_a - D_b) from the lower end a (the
// other coordinates a_k vs), all in round-to-nearest FP64 with no contraction so every build
// places it identically.  As a G-GPDF training point it is rounded to float32 and belongs to
// the voxel that float32 point falls in (always one of the two ends), hence to that voxel's
// leaf.  Marching cubes covers the cells whose lower corner is in a selected leaf and whose 8
// corners are known; the per-case triangles come from a table built on the host by walking
// each cell's faces (see build_mc_table).
//
// Launch shape: one CTA of 512 threads per selected leaf, thread = voxel of the leaf, the
// neighbour leaves looked up once per CTA into shared memory.  Each kernel runs twice: a count
// pass (per-leaf totals, scanned on the device) and an emit pass that writes each leaf's
// records into its own segment in a fixed in-leaf order (voxel bit, then slot / triangle), so
// the output is deterministic up to the order of the leaf segments.
#include <algorithm>

#include "common.cuh"
#include "mesh.h"

namespace vgp {

namespace {

__device__ __forceinline__ int pool_of(const GridView& g, int lx, int ly, int lz) {
    int64_t s = ht_find(g.keys, g.mask, pack_key(lx, ly, lz));
    return s < 0 ? -1 : g.slot2pool[s];
}

__device__ __forceinline__ bool vox_known(const GridView& g, int p, int bit) {
    return p >= 0 && ((g.known[(int64_t)p * 8 + (bit >> 6)] >> (bit & 63)) & 1ull);
}

// zero crossing on the edge from voxel a along `axis` (ends' values Da, Db)
__device__ __forceinline__ void crossing_point(const int a[3], int axis, double Da, double Db, double vs,
                                               double p[3]) {
    const double t = __ddiv_rn(Da, __dsub_rn(Da, Db));
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = __dmul_rn((double)a[k], vs);
    p[axis] = __dmul_rn(__dadd_rn((double)a[axis], t), vs);
}

// fused properties at a crossing: C_a + t (C_b - C_a) per channel with the crossing's t, NaN
// unless both ends hold properties (round-to-nearest, no contraction)
__device__ __forceinline__ void crossing_props(const GridView& g, int64_t ea, int64_t eb, double Da, double Db,
                                               double* out) {
    const double t = __ddiv_rn(Da, __dsub_rn(Da, Db));
    const bool ok = !isnan(g.W[ea]) && !isnan(g.W[eb]);
    for (int ch = 0; ch < g.nc; ++ch) {
        const double ca = g.C[ea * g.nc + ch], cb = g.C[eb * g.nc + ch];
        out[ch] = ok ? __dadd_rn(ca, __dmul_rn(t, __dsub_rn(cb, ca))) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

// Block-wide exclusive prefix sum of small non-negative counts.
__device__ __forceinline__ int block_excl_sum(int v, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int off = 0;
    total = 0;
    for (int w = 0; w < nw; ++w) {
        const int t = wsum[w];
        if (w < wid) off += t;
        total += t;
    }
    __syncthreads();
    return off + x - v;
}

__global__ void k_leaf_list(const uint64_t* gkeys, int64_t cap, const int32_t* slot2pool, const int32_t* flags,
                            int active_only, int32_t* lpool, uint64_t* lkey, int* count) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= cap) return;
    const uint64_t k = gkeys[s];
    if (k == kEmpty) return;
    const int p = slot2pool[s];
    if (p < 0 || (active_only && !(flags[p] & 1))) return;
    const int o = atomicAdd(count, 1);
    lpool[o] = p;
    lkey[o] = k;
}

// The crossing of slot s = 2 axis + (neighbour on the + side) of this thread's voxel, if it
// exists and this voxel owns it.
struct VoxCtx {
    int p, bit, l[3], v[3];
    double Dv;
};

__device__ __forceinline__ bool slot_crossing(const GridView& g, const int* nb, const VoxCtx& c, int s, double vs,
                                              float out[3], double* prop = nullptr) {
    const int axis = s >> 1, dir = (s & 1) ? 1 : -1;
    const int stride = axis == 0 ? 1 : (axis == 1 ? 8 : 64);
    int lc = c.l[axis] + dir, q = c.p;
    if (lc < 0 || lc > 7) {
        q = nb[s];
        lc &= 7;
    }
    const int nbit = c.bit + (lc - c.l[axis]) * stride;
    if (!vox_known(g, q, nbit)) return false;
    const double Dn = g.D[(int64_t)q * 512 + nbit];
    const double Dlo = dir > 0 ? c.Dv : Dn, Dhi = dir > 0 ? Dn : c.Dv;
    if ((Dlo < 0.0) == (Dhi < 0.0)) return false;
    int a[3] = {c.v[0], c.v[1], c.v[2]};
    if (dir < 0) a[axis] -= 1;
    double pd[3];
    crossing_point(a, axis, Dlo, Dhi, vs, pd);
    out[0] = __double2float_rn(pd[0]);
    out[1] = __double2float_rn(pd[1]);
    out[2] = __double2float_rn(pd[2]);
    int i, j, k;
    if (!voxel_ijk(out[0], out[1], out[2], vs, i, j, k)) return false;
    if (!(i == c.v[0] && j == c.v[1] && k == c.v[2])) return false;
    if (prop) {
        const int64_t ev = (int64_t)c.p * 512 + c.bit, en = (int64_t)q * 512 + nbit;
        crossing_props(g, dir > 0 ? ev : en, dir > 0 ? en : ev, Dlo, Dhi, prop);
    }
    return true;
}

template <bool kEmit>
__global__ void __launch_bounds__(512) k_crossings(GridView g, const int32_t* lpool, const uint64_t* lkey, double vs,
                                                   int64_t* cnt, const int64_t* off, int64_t base, float* xyz,
                                                   uint64_t* owner, uint8_t* slot, double* xprop) {
    __shared__ int nb[6];
    __shared__ int wsum[16];
    const int li = blockIdx.x;
    VoxCtx c;
    c.p = lpool[li];
    c.bit = threadIdx.x;
    int LX, LY, LZ;
    unpack_key(lkey[li], LX, LY, LZ);
    if (threadIdx.x < 6) {
        int d[3] = {0, 0, 0};
        d[threadIdx.x >> 1] = (threadIdx.x & 1) ? 1 : -1;
        nb[threadIdx.x] = pool_of(g, LX + d[0], LY + d[1], LZ + d[2]);
    }
    __syncthreads();
    c.l[0] = c.bit & 7;
    c.l[1] = (c.bit >> 3) & 7;
    c.l[2] = c.bit >> 6;
    c.v[0] = 8 * LX + c.l[0];
    c.v[1] = 8 * LY + c.l[1];
    c.v[2] = 8 * LZ + c.l[2];
    const bool known = vox_known(g, c.p, c.bit);
    c.Dv = known ? g.D[(int64_t)c.p * 512 + c.bit] : 0.0;
    int n = 0;
    float tmp[3];
    if (known)
        for (int s = 0; s < 6; ++s) n += slot_crossing(g, nb, c, s, vs, tmp) ? 1 : 0;
    int total;
    const int o = block_excl_sum(n, wsum, total);
    if (!kEmit) {
        if (threadIdx.x == 0) cnt[li] = total;
        return;
    }
    if (n == 0) return;
    int64_t w = base + off[li] + o;
    const uint64_t okey = pack_key(c.v[0], c.v[1], c.v[2]);
    for (int s = 0; s < 6; ++s) {
        if (!slot_crossing(g, nb, c, s, vs, tmp, xprop ? xprop + w * g.nc : nullptr)) continue;
        xyz[3 * w] = tmp[0];
        xyz[3 * w + 1] = tmp[1];
        xyz[3 * w + 2] = tmp[2];
        if (owner) owner[w] = okey;
        if (slot) slot[w] = (uint8_t)s;
        ++w;
    }
}

template <bool kEmit>
__global__ void __launch_bounds__(512) k_mesh(GridView g, const int32_t* lpool, const uint64_t* lkey,
                                              const uint8_t* tab, const uint8_t* ntri, double vs, int64_t* cnt,
                                              const int64_t* off, double* xyz, uint64_t* ekey, uint8_t* eaxis,
                                              double* vprop) {
    __shared__ int nb[8];
    __shared__ int wsum[16];
    const int li = blockIdx.x, b = threadIdx.x;
    int LX, LY, LZ;
    unpack_key(lkey[li], LX, LY, LZ);
    if (b < 8) nb[b] = b == 0 ? lpool[li] : pool_of(g, LX + (b & 1), LY + ((b >> 1) & 1), LZ + (b >> 2));
    __syncthreads();
    const int l0 = b & 7, l1 = (b >> 3) & 7, l2 = b >> 6;
    double D[8];
    int64_t E[8];  // pool element of each corner
    int mask = 0;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cx = l0 + (c & 1), cy = l1 + ((c >> 1) & 1), cz = l2 + (c >> 2);
        const int q = nb[(cx >> 3) + 2 * (cy >> 3) + 4 * (cz >> 3)];
        const int cb = (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7);
        E[c] = (int64_t)q * 512 + cb;
        D[c] = 0.0;
        if (ok && vox_known(g, q, cb)) {
            D[c] = g.D[(int64_t)q * 512 + cb];
            if (D[c] < 0.0) mask |= 1 << c;
        } else {
            ok = false;
        }
    }
    const int nt = ok ? (int)ntri[mask] : 0;
    int total;
    const int o = block_excl_sum(nt, wsum, total);
    if (!kEmit) {
        if (b == 0) cnt[li] = total;
        return;
    }
    const int v[3] = {8 * LX + l0, 8 * LY + l1, 8 * LZ + l2};
    for (int t = 0; t < nt; ++t) {
        const int64_t w = off[li] + o + t;
        for (int j = 0; j < 3; ++j) {
            const int e = tab[mask * 16 + 3 * t + j];
            const int axis = e >> 2, u = (axis + 1) % 3, ww = (axis + 2) % 3;
            const int lc = ((e & 1) << u) | (((e >> 1) & 1) << ww);
            const int uc = lc | (1 << axis);
            const int a[3] = {v[0] + (lc & 1), v[1] + ((lc >> 1) & 1), v[2] + (lc >> 2)};
            double p[3];
            crossing_point(a, axis, D[lc], D[uc], vs, p);
            xyz[9 * w + 3 * j] = p[0];
            xyz[9 * w + 3 * j + 1] = p[1];
            xyz[9 * w + 3 * j + 2] = p[2];
            ekey[3 * w + j] = pack_key(a[0], a[1], a[2]);
            eaxis[3 * w + j] = (uint8_t)axis;
            if (vprop) crossing_props(g, E[lc], E[uc], D[lc], D[uc], vprop + (3 * w + j) * g.nc);
        }
    }
}

// keep[i] = 1 unless point i lies in a leaf that the latest fusion touched
__global__ void k_store_keep(const float* pts, int64_t n, double vs, GridView g, const int32_t* flags, int64_t* keep) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int x, y, z;
    int k = 1;
    if (voxel_ijk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], vs, x, y, z)) {
        const int p = pool_of(g, leaf_coord(x), leaf_coord(y), leaf_coord(z));
        if (p >= 0 && (flags[p] & 1)) k = 0;
    }
    keep[i] = k;
}

__global__ void k_store_compact(const float* pts, int64_t n, const int64_t* keep, const int64_t* pos, float* out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    const int64_t o = pos[i];
    out[3 * o] = pts[3 * i];
    out[3 * o + 1] = pts[3 * i + 1];
    out[3 * o + 2] = pts[3 * i + 2];
}

constexpr int TB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TB - 1) / TB); }

}  // namespace

// Marching-cubes triangles of all 256 inside masks.  Corner c = x + 2 y + 4 z of the cell;
// a cell edge is named by its lower corner and axis; in the table it is stored as
// 4 axis + bit_u + 2 bit_w (u = axis + 1, w = axis + 2 mod 3: the lower corner's other two
// coordinates).  Each face is walked counter-clockwise seen from outside the cell; an edge
// leaving an inside corner for an outside one links to the edge that enters the run of
// inside corners behind it, so inside corners that meet only across a face diagonal stay
// apart and the two cells sharing a face resolve it alike.  The links form loops; each
// loop is taken from its first edge in (lower corner, axis) order and fanned in reverse,
// which turns the normals towards increasing D.
void build_mc_table(uint8_t* tab, uint8_t* ntri) {
    auto tab_edge = [](int c0, int c1) {
        const int d = c0 ^ c1;
        const int axis = d == 1 ? 0 : (d == 2 ? 1 : 2);
        const int lo = std::min(c0, c1);
        const int u = (axis + 1) % 3, w = (axis + 2) % 3;
        return 4 * axis + ((lo >> u) & 1) + 2 * ((lo >> w) & 1);
    };
    // (lower corner, axis) order of the 12 edges, as table edges
    int order[12], no = 0;
    for (int lc = 0; lc < 8; ++lc)
        for (int axis = 0; axis < 3; ++axis)
            if (!((lc >> axis) & 1)) order[no++] = tab_edge(lc, lc | (1 << axis));
    static const int ring[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
    for (int mask = 0; mask < 256; ++mask) {
        auto in = [mask](int c) { return (mask >> c) & 1; };
        int link[12];
        std::fill(link, link + 12, -1);
        for (int axis = 0; axis < 3; ++axis) {
            const int u = (axis + 1) % 3, w = (axis + 2) % 3;
            for (int side = 0; side < 2; ++side) {
                int q[4];
                for (int i = 0; i < 4; ++i) {
                    const int r = side ? i : (4 - i) & 3;  // the -axis face runs the ring backwards
                    q[i] = (side << axis) | (ring[r][0] << u) | (ring[r][1] << w);
                }
                for (int k = 0; k < 4; ++k) {
                    if (!in(q[k]) || in(q[(k + 1) & 3])) continue;
                    int j = k;
                    while (in(q[(j + 3) & 3])) j = (j + 3) & 3;
                    link[tab_edge(q[k], q[(k + 1) & 3])] = tab_edge(q[(j + 3) & 3], q[j]);
                }
            }
        }
        bool used[12] = {};
        int nt = 0;
        for (int oi = 0; oi < 12; ++oi) {
            const int e0 = order[oi];
            if (link[e0] < 0 || used[e0]) continue;
            int loop[12], m = 0;
            for (int e = e0; !used[e]; e = link[e]) {
                used[e] = true;
                loop[m++] = e;
            }
            for (int i = 1; i + 1 < m; ++i) {
                tab[mask * 16 + 3 * nt] = (uint8_t)loop[0];
                tab[mask * 16 + 3 * nt + 1] = (uint8_t)loop[i + 1];
                tab[mask * 16 + 3 * nt + 2] = (uint8_t)loop[i];
                ++nt;
            }
        }
        ntri[mask] = (uint8_t)nt;
    }
}

void mesh_leaf_list(const GridView& g, const int32_t* flags, int active_only, int32_t* lpool, uint64_t* lkey,
                    int* count, cudaStream_t st) {
    const int64_t cap = (int64_t)g.mask + 1;
    k_leaf_list<<<nblk(cap), TB, 0, st>>>(g.keys, cap, g.slot2pool, flags, active_only, lpool, lkey, count);
    note_launch();
}

void mesh_crossings(const GridView& g, const int32_t* lpool, const uint64_t* lkey, int nl, double vs, int64_t* cnt,
                    const int64_t* off, int64_t base, float* xyz, uint64_t* owner, uint8_t* slot, double* xprop,
                    bool emit, cudaStream_t st) {
    if (nl <= 0) return;
    if (emit)
        k_crossings<true><<<nl, 512, 0, st>>>(g, lpool, lkey, vs, cnt, off, base, xyz, owner, slot, xprop);
    else
        k_crossings<false><<<nl, 512, 0, st>>>(g, lpool, lkey, vs, cnt, off, base, xyz, owner, slot, nullptr);
    note_launch();
}

void mesh_triangles(const GridView& g, const int32_t* lpool, const uint64_t* lkey, int nl, const uint8_t* tab,
                    const uint8_t* ntri, double vs, int64_t* cnt, const int64_t* off, double* xyz, uint64_t* ekey,
                    uint8_t* eaxis, double* vprop, bool emit, cudaStream_t st) {
    if (nl <= 0) return;
    if (emit)
        k_mesh<true><<<nl, 512, 0, st>>>(g, lpool, lkey, tab, ntri, vs, cnt, off, xyz, ekey, eaxis, vprop);
    else
        k_mesh<false><<<nl, 512, 0, st>>>(g, lpool, lkey, tab, ntri, vs, cnt, off, xyz, ekey, eaxis, nullptr);
    note_launch();
}

void store_keep(const float* pts, int64_t n, double vs, const GridView& g, const int32_t* flags, int64_t* keep,
                cudaStream_t st) {
    if (n <= 0) return;
    k_store_keep<<<nblk(n), TB, 0, st>>>(pts, n, vs, g, flags, keep);
    note_launch();
}

void store_compact(const float* pts, int64_t n, const int64_t* keep, const int64_t* pos, float* out,
                   cudaStream_t st) {
    if (n <= 0) return;
    k_store_compact<<<nblk(n), TB, 0, st>>>(pts, n, keep, pos, out);
    note_launch();
}

}  // namespace vgp
