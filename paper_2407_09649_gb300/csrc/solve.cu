// solve.cu -- batched GP instances: K assembly, FP64 Cholesky, alpha, and the fused
// evaluation of every query of the instance (latent mean Eq. 1, variance Eq. 2, gradient
// Eq. 5, reverting Eq. 3 and distance variance Eq. 4), plus the backward pass.
//
// One CTA owns one instance at a time and pulls instances from a list sorted by decreasing
// size (a persistent launch per size bucket, longest first).  A = K + sigma^2 I is stored as
// the lower triangle of 8x8 tiles (64 contiguous doubles per tile, tiles in packed row
// order), in shared memory when it fits, else in a per-CTA global workspace.  The Cholesky
// factorisation is right-looking by 8-column panels; the panel solve and the trailing
// update run on the FP64 tensor path (mma.sync m8n8k4 f64), the 8x8 diagonal blocks on the
// FP64 pipe.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "internal.h"

namespace vgp {

namespace {

// offset of tile (it, jt), jt <= it, in the tile-packed lower triangle
__host__ __device__ __forceinline__ int64_t tix(int it, int jt) { return ((int64_t)it * (it + 1) / 2 + jt) * 64; }
__host__ __device__ __forceinline__ int64_t n_tiles(int nt) { return (int64_t)nt * (nt + 1) / 2; }

// Position of element (r, c) inside a 64-double tile: row major with the columns of rows
// 2, 3, 6, 7 XOR-swizzled by 4, so the mma fragment loads (row g, column t) of the 32 lanes
// of a warp hit distinct shared-memory banks in each half-warp.
__host__ __device__ __forceinline__ int te(int r, int c) { return r * 8 + (c ^ ((r & 2) << 1)); }

// row index of packed-triangle entry p (0 <= col <= row)
__device__ __forceinline__ int tri_row(int p) {
    int r = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= p) ++r;
    while (r * (r + 1) / 2 > p) --r;
    return r;
}

__device__ __forceinline__ double neg(double x) {  // sign flip on the integer pipe
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// D(8x8) += A(8x4) B(4x8) on the FP64 tensor path.  Fragments: a = A[g][t],
// b = B[t][g], c = D[g][2t .. 2t+1] with g = lane / 4, t = lane % 4.
__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c0), "+d"(c1)
                 : "d"(a), "d"(b));
}

constexpr int kEmuThreads = 256;  // CTA size of the emulated-update kernels (two CTAs per SM)
constexpr int kEB = 4;            // tiles (of 8 columns) per block of the emulated factorisation
constexpr int kEK = kEB / 2;      // 16-column mma steps per block

struct SolveCtx {
    SolveBatch b;
    DevParams P;
    int* err;
    int* counter;
    const int32_t* order;  // instance ids, decreasing N (null: inst_base + work index)
    int inst_base;
    int n_work;
    const int* plan;       // device bucket plan (graph mode): counts [5], then offsets [5]
    int bucket;
    int npad;              // largest N in this launch, rounded up to 8
    int a_in_smem;
    int stage_panel;       // A global: current panel column staged in shared memory
    double* ws_a;          // per-CTA tile-packed A when not in shared memory
    int64_t ws_a_stride;
    double* ws_v;          // per-CTA variance columns [npad][blockDim]
    int64_t ws_v_stride;
    uint8_t* ws_e;         // per-CTA bf16 slices and row scales (emulated trailing updates)
    int64_t ws_e_stride;
    BackwardBatch bw;
    const int* chunk_off = nullptr;  // work items (see k_chunk_plan): chunk offsets over the order;
                                     // nullptr: one work item per instance
    const int* chunk_q = nullptr;    // queries of a work item for this launch (0: all of them)
    int qmax = 0;          // emulated kernel with variance: query rows appended to A (0: none)
    int nrow = 0;          // emulated kernel: rows of the workspace matrices (npad + qmax)
};

struct Shared {
    double* X;      // [N][3] local FP64
    double* alpha;  // [npad]
    double* invd;   // [npad] 1 / L_ii
    double* z;      // [npad] scratch
    double* w;      // [npad] scratch (backward pass only)
    double* Tinv;   // [64] inverse of the current diagonal tile
    double* T256;   // [256] 2^(j/256) for exp_neg
    double* A;      // tile-packed lower triangle
    double* panel;  // [npad/8 - 1][64] current panel column when A is in global memory
    float* Xf;      // [N][3]
    float* alf;     // [npad] alpha rounded to FP32
    float* alf_lo;  // [npad] alpha - alf, rounded to FP32
    int* xi;        // [npad] lattice offsets x | y << 8 | z << 16 (lattice instances)
    double* pa[4];  // property weights per channel (property mode): channels 0 and 1 reuse the
                    // distance alpha and its FP32 copies, which that mode does not use
    double* Tblk;   // [kEB][64] inverses of the diagonal tiles of the current block
    double* Wsc;    // [warps][64] per-warp tile scratch (layout changes between mma operands)
    unsigned char* stage;  // emulated kernel: slice operands of the tensor-core updates (aliases
                           // X .. alf_lo, which the factorisation does not use; reloaded after it)
    float* qw;             // emulated kernel: [kBorderQ][3] world coordinates of appended queries (FP32;
                           // NaN: not finite); lattice instances: [0] the lattice code's bits, [1] NaN
                           // when not finite
    float* Xw;             // emulated kernel: [npad][3] world coordinates of the points (FP32, exact)
    float2* Tff;           // emulated kernel: 2^(j/256), j = 0..255, as float pairs
};

// Emulated trailing updates on the tensor cores (tcgen05): an output tile is kBandT row tiles
// (128 rows, the MMA's M) by kColT row tiles (32 columns, its N) of the trailing matrix; the
// slices of one 16-column half of the block are staged for the band (A) and the column tile (B).
constexpr int kBandT = 16;
constexpr int kColT = 4;
constexpr int kSliceTileBytes = 7 * 2 * 128;  // one row tile, one K half: 7 slices x 2 core matrices
// staging: the band's slices of both K halves (A), and two buffers of the column tile's (B)
constexpr int kStageA = 2 * kBandT * kSliceTileBytes;
constexpr int kStageB = 2 * kColT * kSliceTileBytes;
constexpr int kStageBytes = kStageA + 2 * kStageB;
constexpr int kEmuTmemCols = 8 * 8 * kColT;    // 8 slice groups x 32 FP32 columns
// Latent variance in the emulated kernel: up to kBorderQ queries of an instance append their
// kernel vectors to A as rows, so the factorisation itself yields 1 - |L^-1 k|^2 (see
// fit_instance); an instance with more queries is factorised once per chunk of kBorderQ.
// Instances gather the queries of several query leaves (those that fall back to a shared
// leaf), so the bound is set high: a factorisation costs about N^3/6 products against
// N^2/2 per appended row.
constexpr int kBorderQ = 1024;
constexpr int kEmuCtasPerSm = 512 / kEmuTmemCols;  // CTAs whose tensor memory fits one SM

__host__ __device__ __forceinline__ size_t align128(size_t x) { return (x + 127) & ~(size_t)127; }
__host__ __device__ __forceinline__ size_t emu_fixed_bytes(int npad) {
    // invd, T256, Tblk, Wsc, Tff
    return align128((size_t)(npad + 256 + kEB * 64 + 8 * 64 + 256) * sizeof(double));
}
__host__ __device__ __forceinline__ size_t emu_point_bytes(int npad, int nprop, bool lattice) {
    return (size_t)5 * npad * sizeof(double) + (size_t)5 * npad * sizeof(float) +
           (lattice ? (size_t)npad * sizeof(int) : 0) + (size_t)(nprop > 2 ? nprop - 2 : 0) * npad * sizeof(double);
}
// the points (also as FP32 world coordinates) and the appended queries (both forms)
__host__ __device__ __forceinline__ size_t emu_alias_bytes(int npad, int nprop, bool lattice) {
    const size_t b = emu_point_bytes(npad, nprop, lattice) + (lattice ? 0 : (size_t)3 * npad * sizeof(float)) +
                     (size_t)kBorderQ * 3 * sizeof(float);
    return b > (size_t)kStageBytes ? b : (size_t)kStageBytes;
}

// Emulated kernel: invd, the exp table, the block's tile inverses and the warp scratch first, then
// (128-byte aligned) the staging buffer of the tensor-core updates, which X, alpha, z, Xf, alf,
// alf_lo, xi and the property weights alias.
__device__ Shared carve_emu(double* sm, int npad, double* ws_a, int nprop, bool lattice) {
    Shared s;
    s.invd = sm;
    s.T256 = s.invd + npad;
    s.Tblk = s.T256 + 256;
    s.Wsc = s.Tblk + kEB * 64;
    s.Tinv = nullptr;
    s.w = nullptr;
    s.panel = nullptr;
    s.A = ws_a;
    s.stage = reinterpret_cast<unsigned char*>(sm) + emu_fixed_bytes(npad);
    s.X = reinterpret_cast<double*>(s.stage);
    s.alpha = s.X + 3 * npad;
    s.z = s.alpha + npad;
    s.Xf = reinterpret_cast<float*>(s.z + npad);
    s.alf = s.Xf + 3 * npad;
    s.alf_lo = s.alf + npad;
    s.xi = lattice ? reinterpret_cast<int*>(s.alf_lo + npad) : nullptr;
    double* extra = reinterpret_cast<double*>(reinterpret_cast<int*>(s.alf_lo + npad) + (lattice ? npad : 0));
    s.pa[0] = s.alpha;
    s.pa[1] = reinterpret_cast<double*>(s.alf);
    s.pa[2] = nprop > 2 ? extra : nullptr;
    s.pa[3] = nprop > 3 ? extra + npad : nullptr;
    // world coordinates of the points off the lattice only (lattice values come from tables)
    float* after = reinterpret_cast<float*>(s.stage + emu_point_bytes(npad, nprop, lattice));
    s.Xw = lattice ? nullptr : after;
    s.qw = lattice ? after : after + 3 * npad;
    s.Tff = reinterpret_cast<float2*>(s.Wsc + 8 * 64);
    return s;
}

__device__ Shared carve(double* sm, int npad, int a_in_smem, double* ws_a, int nprop, int stage_panel,
                        bool lattice, bool with_w, bool emu = false) {
    if (emu) return carve_emu(sm, npad, ws_a, nprop, lattice);
    Shared s;
    s.stage = nullptr;
    s.qw = nullptr;
    s.Xw = nullptr;
    s.Tff = nullptr;
    s.X = sm;
    s.alpha = s.X + 3 * npad;
    s.invd = s.alpha + npad;
    s.z = s.invd + npad;
    s.w = with_w ? s.z + npad : nullptr;
    s.Tinv = s.z + (with_w ? 2 : 1) * npad;
    s.T256 = s.Tinv + 64;
    double* end = s.T256 + 256;
    s.Tblk = nullptr;
    s.Wsc = nullptr;
    if (a_in_smem) {
        s.A = end;
        end += n_tiles(npad / 8) * 64;
        s.panel = nullptr;
    } else {
        s.A = ws_a;
        s.panel = stage_panel ? end : nullptr;
        if (stage_panel) end += (int64_t)(npad / 8) * 64;
    }
    s.Xf = reinterpret_cast<float*>(end);
    s.alf = s.Xf + 3 * npad;
    s.alf_lo = s.alf + npad;
    s.xi = lattice ? reinterpret_cast<int*>(s.alf_lo + npad) : nullptr;
    double* extra = reinterpret_cast<double*>(reinterpret_cast<int*>(s.alf_lo + npad) + (lattice ? npad : 0));
    // (4 npad bytes of xi keep 8-byte alignment: npad is a multiple of 8)
    s.pa[0] = s.alpha;
    s.pa[1] = reinterpret_cast<double*>(s.alf);  // alf, alf_lo: 2 npad floats, 8-byte aligned
    s.pa[2] = nprop > 2 ? extra : nullptr;
    s.pa[3] = nprop > 3 ? extra + npad : nullptr;
    return s;
}

__host__ size_t smem_bytes(int npad, int a_in_smem, int nprop, int stage_panel, bool lattice, bool with_w = false,
                          bool emu = false) {
    if (emu) return emu_fixed_bytes(npad) + emu_alias_bytes(npad, nprop, lattice);
    size_t d = (size_t)(with_w ? 7 : 6) * npad + 64 + 256 +
               (a_in_smem ? (size_t)n_tiles(npad / 8) * 64 : (stage_panel ? (size_t)(npad / 8) * 64 : 0));
    return d * sizeof(double) + (size_t)5 * npad * sizeof(float) + (lattice ? (size_t)npad * sizeof(int) : 0) +
           (size_t)std::max(nprop - 2, 0) * npad * sizeof(double);
}

__device__ __forceinline__ int lat_m(int a, int b) {
    const int dx = (a & 255) - (b & 255), dy = ((a >> 8) & 255) - ((b >> 8) & 255), dz = ((a >> 16) & 255) - ((b >> 16) & 255);
    return dx * dx + dy * dy + dz * dz;
}

// SE kernel value of a pair of training points (Sec. III-A), FP64: from the exact lattice
// table for voxel-centre instances, else exp_neg (mixed) or the library exp (plain).
__device__ __forceinline__ double kval_pair(const DevParams& P, const Shared& s, bool lattice, int i, int j) {
    if (lattice) return P.lat_tab[lat_m(s.xi[i], s.xi[j])];
    double dx = s.X[3 * i] - s.X[3 * j], dy = s.X[3 * i + 1] - s.X[3 * j + 1], dz = s.X[3 * i + 2] - s.X[3 * j + 2];
    const double y = -(dx * dx + dy * dy + dz * dz) * P.inv2l2;
    return P.precision == VGP_MIXED ? exp_neg(y, s.T256) : exp(y);
}

// ---- the emulated kernel's matrix in fixed point -------------------------------------------
// Until its column block is reached, an entry of the emulated factorisation is held as the
// integer round(v 2^61) (|v| <= 1 + sigma^2: every entry of K + sigma^2 I and of its Schur
// complements is bounded by the largest diagonal entry).  The trailing updates then subtract
// integers (one shift and one 64-bit subtraction per entry) and the block's columns are
// turned into FP64 once, by the update that completes them.  Resolution 2^-61, far below the
// updates' own rounding (2^-55 of the row maxima).
constexpr int kFixBits = 61;
__device__ __forceinline__ long long fix_of_double(double v) { return __double2ll_rn(v * 0x1p61); }
// f 2^-61 as FP64: the conversion, then the exponent lowered by 61 on the integer pipe
// (|f| >= 1 keeps the result normal)
__device__ __forceinline__ double double_of_fix(long long f) {
    return f == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(__ll2double_rn(f)) - (61ll << 52));
}

// round(x 2^e) of a float x, |x| 2^e < 2^62, on the integer pipe (ties away from zero; 0 for
// subnormal x).
__device__ __forceinline__ long long fix_of_float(float x, int e) {
    const unsigned b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 255);
    if (ex == 0) return 0;
    const long long mant = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = ex - 150 + e;  // |x| = mant 2^(ex - 150)
    long long v;
    if (sh >= 0)
        v = mant << sh;
    else if (sh >= -25)
        v = ((mant >> (-sh - 1)) + 1) >> 1;
    else
        v = 0;
    return (b >> 31) ? -v : v;
}

// Float pairs: a value is hi + lo, |lo| near 2^-24 |hi| at most.  Knuth's two-sum and the
// FMA product error are error-free; every operation is an _rn intrinsic, so nothing is
// contracted or reassociated.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// ln2/256 = kL0 + kL1 + kL2 (kL0 with 10 significant bits, so n kL0 is exact for n < 2^14;
// the three parts hold 58 bits) and 256/ln2.
constexpr float kL0 = 0x1.63p-9f, kL1 = -0x1.bd0106p-21f, kL2 = 0x1.cf79acp-48f;
constexpr float kInvL = 369.32993046757464f;

// k = exp(-|a - b|^2 / (2 l^2)) in the fixed point above, on the FP32 and integer pipes (the
// mixed-precision entries of the emulated kernel; the FP64 pipe is the scarce unit of the
// factorisation).  a, b: FP32 world coordinates (the inputs' own values), so each difference
// is exactly a float pair (two-sum) and |a - b|^2 is carried as a float pair renormalised
// after every axis;
//   y = |a - b|^2 / (2 l^2) as a float pair;
//   e^-y = 2^-(n/256) e^r with n = round(256 y / ln2) and r = n ln2/256 - y, |r| <= ln2/512
//   (Tang's table-driven reduction, as exp_neg), r as a normalised float pair, e^r from its
//   Taylor terms to r^4 (the next term is below 2^-54), 2^(i/256) from the float-pair table;
//   the float-pair result scaled by 2^(61 - m) into a 64-bit integer.
// The error stays below 2^-45 k (1 + y) + 2 units of 2^-61, about 2^-47 at most in k, at the
// level of the Cholesky's own backward error; 0 where y > 43.5 (k < 2^-62).
__device__ __forceinline__ long long kfix_ff(const float a[3], const float b[3], float ch, float cl,
                                             const float2* tab) {
    float S = 0.f, E = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float dh, dl;
        two_sum(a[k], -b[k], dh, dl);  // a - b = dh + dl exactly
        const float p = __fmul_rn(dh, dh), pe = __fmaf_rn(dh, dh, -p);
        float t, te;
        two_sum(S, p, t, te);
        // (dh + dl)^2 = p + pe + dl (2 dh + dl); then renormalise (S, E)
        E = __fadd_rn(E, __fadd_rn(te, __fmaf_rn(dl, __fmaf_rn(2.f, dh, dl), pe)));
        S = __fadd_rn(t, E);
        E = __fsub_rn(E, __fsub_rn(S, t));
    }
    const float yh = __fmul_rn(S, ch);
    const float yl = __fadd_rn(__fmaf_rn(S, ch, -yh), __fmaf_rn(S, cl, __fmul_rn(E, ch)));
    if (!(yh <= 43.5f)) return 0;
    const float n = rintf(__fmul_rn(yh, kInvL));
    const int ni = (int)n;
    // r = (n kL0 - yh) + n kL1 - yl + n kL2, the large parts summed error-free
    float a0, ae, b0, be, rh, ce;
    two_sum(__fmul_rn(n, kL0), -yh, a0, ae);
    const float p2 = __fmul_rn(n, kL1), p2e = __fmaf_rn(n, kL1, -p2);
    two_sum(a0, p2, b0, be);
    two_sum(b0, -yl, rh, ce);
    const float rl = __fadd_rn(__fadd_rn(__fadd_rn(ae, be), ce), __fmaf_rn(n, kL2, p2e));
    // e^r - 1 = rh + rh^2/2 + [rl + rh rl + rh^3/6 + rh^4/24 + (rh^2 error)/2]
    const float q = __fmul_rn(rh, rh), qe = __fmaf_rn(rh, rh, -q);
    const float c34 = __fmul_rn(__fmul_rn(q, rh), __fmaf_rn(rh, 1.f / 24.f, 1.f / 6.f));
    const float small = __fadd_rn(__fmaf_rn(0.5f, qe, rl), __fmaf_rn(rh, rl, c34));
    float u, ue, eh, e4;
    two_sum(rh, __fmul_rn(0.5f, q), u, ue);
    two_sum(1.f, u, eh, e4);
    const float el = __fadd_rn(e4, __fadd_rn(ue, small));
    // 2^(-n/256) = 2^-m 2^(i/256) with m = ceil(n / 256) and i = (-n) mod 256
    const int j = ni & 255, m = (ni >> 8) + (j != 0);
    const float2 T = tab[(256 - j) & 255];
    const float vh = __fmul_rn(T.x, eh);
    const float vl = __fadd_rn(__fmaf_rn(T.x, eh, -vh), __fmaf_rn(T.x, el, __fmul_rn(T.y, eh)));
    return fix_of_float(vh, kFixBits - m) + fix_of_float(vl, kFixBits - m);
}

// Entry (i, j), i > j, of K in the fixed point: float pairs in mixed precision, the FP64 value
// (as kval_pair) rounded to the fixed point in FP64 precision and on the lattice.
__device__ __forceinline__ long long kfix_pair(const DevParams& P, const Shared& s, bool lattice, int i, int j) {
    if (lattice || P.precision != VGP_MIXED) return fix_of_double(kval_pair(P, s, lattice, i, j));
    return kfix_ff(s.Xw + 3 * i, s.Xw + 3 * j, P.inv2l2_hi, P.inv2l2_lo, s.Tff);
}

// The float pair (hi, lo) of an FP64 value.
__device__ __forceinline__ void split_pair(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Solve (L L^T) x = rhs in place on s.z (x written to out), L tile-packed; rows >= N of rhs
// must be zero.  Right-looking by 8-row blocks on each side.
__device__ void chol_solve(const Shared& s, const double* A, int Nt, double* out) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Np = Nt * 8;
    double* z = s.z;
    for (int kt = 0; kt < Nt; ++kt) {
        if (tid == 0) {
            const double* D = A + tix(kt, kt);
            for (int r = 0; r < 8; ++r) {
                double v = z[8 * kt + r];
                for (int c2 = 0; c2 < r; ++c2) v -= D[te(r, c2)] * z[8 * kt + c2];
                z[8 * kt + r] = v * s.invd[8 * kt + r];
            }
        }
        __syncthreads();
        for (int i = 8 * (kt + 1) + tid; i < Np; i += nt) {
            const double* T = A + tix(i >> 3, kt);
            const int r = i & 7;
            double v = z[i];
#pragma unroll
            for (int c2 = 0; c2 < 8; ++c2) v -= T[te(r, c2)] * z[8 * kt + c2];
            z[i] = v;
        }
        __syncthreads();
    }
    for (int kt = Nt - 1; kt >= 0; --kt) {
        if (tid == 0) {
            const double* D = A + tix(kt, kt);
            for (int r = 7; r >= 0; --r) {
                double v = z[8 * kt + r];
                for (int c2 = r + 1; c2 < 8; ++c2) v -= D[te(c2, r)] * out[8 * kt + c2];
                out[8 * kt + r] = v * s.invd[8 * kt + r];
            }
        }
        __syncthreads();
        for (int j = tid; j < 8 * kt; j += nt) {
            const double* T = A + tix(kt, j >> 3);
            const int cj = j & 7;
            double v = z[j];
#pragma unroll
            for (int c2 = 0; c2 < 8; ++c2) v -= T[te(c2, cj)] * out[8 * kt + c2];
            z[j] = v;
        }
        __syncthreads();
    }
}

// Solve (L L^T) x = rhs in place on s.z (x written to out) with the inverses of every diagonal
// tile in Tall ([Nt][64], tile layout); rows >= N of rhs must be zero.  Blocks of four tiles:
// inside a block warp 0 alone takes each tile (its inverse times the right-hand side, eight
// lanes) and updates the rest of the block; the rows outside the block are then updated by
// the whole CTA, two barriers per block and side.
__device__ void chol_solve_inv(const Shared& s, const double* A, int Nt, double* out, const double* Tall) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int Np = Nt * 8;
    double* z = s.z;
    for (int B0 = 0; B0 < Nt; B0 += 4) {
        const int B1 = min(B0 + 4, Nt);
        if (tid < 32) {
            for (int kt = B0; kt < B1; ++kt) {
                const double* Ti = Tall + 64 * kt;
                double v = 0.0;
                if (lane < 8)
                    for (int c2 = 0; c2 <= lane; ++c2) v += Ti[te(lane, c2)] * z[8 * kt + c2];
                __syncwarp();
                if (lane < 8) z[8 * kt + lane] = v;
                __syncwarp();
                const int i = 8 * (kt + 1) + lane;  // rows of the block below tile kt
                if (i < 8 * B1) {
                    const double* T = A + tix(i >> 3, kt);
                    const int r = i & 7;
                    double u = z[i];
#pragma unroll
                    for (int c2 = 0; c2 < 8; ++c2) u -= T[te(r, c2)] * z[8 * kt + c2];
                    z[i] = u;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = 8 * B1 + tid; i < Np; i += nt) {
            const int r = i & 7;
            double u = z[i];
            for (int kt = B0; kt < B1; ++kt) {
                const double* T = A + tix(i >> 3, kt);
#pragma unroll
                for (int c2 = 0; c2 < 8; ++c2) u -= T[te(r, c2)] * z[8 * kt + c2];
            }
            z[i] = u;
        }
        __syncthreads();
    }
    for (int B1 = Nt; B1 > 0; B1 -= 4) {
        const int B0 = max(B1 - 4, 0);
        if (tid < 32) {
            for (int kt = B1 - 1; kt >= B0; --kt) {
                const double* Ti = Tall + 64 * kt;
                double v = 0.0;
                if (lane < 8)
                    for (int r = lane; r < 8; ++r) v += Ti[te(r, lane)] * z[8 * kt + r];
                __syncwarp();
                if (lane < 8) out[8 * kt + lane] = v;
                __syncwarp();
                const int j = 8 * B0 + lane;  // columns of the block left of tile kt
                if (j < 8 * kt) {
                    const double* T = A + tix(kt, j >> 3);
                    const int cj = j & 7;
                    double u = z[j];
#pragma unroll
                    for (int c2 = 0; c2 < 8; ++c2) u -= T[te(c2, cj)] * out[8 * kt + c2];
                    z[j] = u;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int j = tid; j < 8 * B0; j += nt) {
            const int cj = j & 7;
            double u = z[j];
            for (int kt = B0; kt < B1; ++kt) {
                const double* T = A + tix(kt, j >> 3);
#pragma unroll
                for (int c2 = 0; c2 < 8; ++c2) u -= T[te(c2, cj)] * out[8 * kt + c2];
            }
            z[j] = u;
        }
        __syncthreads();
    }
}

// One warp: the 8x8 Cholesky of diagonal tile kt in place (right-looking, the column scaling
// and rank-1 updates spread over the lanes, 1 / L_jj from rsqrt), 1 / L_jj into invd and the
// inverse of the tile's factor into Ti (rows by forward substitution, one lane per column).
// S: 64 doubles of scratch.  False on a non-positive pivot (the same on every lane).
__device__ bool diag_tile_warp(double* A, int kt, const Shared& s, double* Ti, double* S) {
    const int lane = threadIdx.x & 31;
    double* D = A + tix(kt, kt);
    S[lane] = D[lane];
    S[lane + 32] = D[lane + 32];
    __syncwarp();
    for (int j = 0; j < 8; ++j) {
        const double v = S[te(j, j)];
        if (!(v > 0.0)) return false;
        const double r = rsqrt(v);
        __syncwarp();
        if (lane > j && lane < 8) S[te(lane, j)] *= r;
        if (lane == 0) {
            S[te(j, j)] = v * r;
            s.invd[8 * kt + j] = r;
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // entries (rr, cc), j < cc <= rr
            const int e = lane + 32 * h, rr = e >> 3, cc = e & 7;
            if (cc > j && rr >= cc) S[te(rr, cc)] -= S[te(rr, j)] * S[te(cc, j)];
        }
        __syncwarp();
    }
    D[lane] = S[lane];
    D[lane + 32] = S[lane + 32];
    // Ti = L^-1: Ti_ii = 1 / L_ii, Ti_ic = -(sum_{c <= k < i} L_ik Ti_kc) / L_ii for c < i
    for (int i = 0; i < 8; ++i) {
        if (lane < 8) {
            double u = lane == i ? 1.0 : 0.0;
            for (int k = lane; k < i; ++k) u -= S[te(i, k)] * Ti[te(k, lane)];
            Ti[te(i, lane)] = lane <= i ? u * s.invd[8 * kt + i] : 0.0;
        }
        __syncwarp();
    }
    return true;
}

// Panel column kt: L_it,kt = A_it,kt Ti^T for kt < it < it_end (Ti: inverse of the diagonal
// tile's factor), one tile per warp.
__device__ void panel_column(double* A, int kt, int it_end, const double* Ti) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int it = kt + 1 + warp; it < it_end; it += nwarps) {
        double* T = A + tix(it, kt);
        const double a0 = T[te(g, t)], a1 = T[te(g, 4 + t)];
        const double b0 = Ti[te(g, t)], b1 = Ti[te(g, 4 + t)];
        double c0 = 0.0, c1 = 0.0;
        dmma(c0, c1, a0, b0);
        dmma(c0, c1, a1, b1);
        __syncwarp();
        T[te(g, 2 * t)] = c0;
        T[te(g, 2 * t + 1)] = c1;
    }
}

// w 2^sh rounded to an integer (ties up) for a 64-bit integer w: a slice-product update in
// the fixed point of the trailing matrix.  No overflow: |w| 2^sh is bounded by the entry bound.
__device__ __forceinline__ long long fix_shift(long long w, int sh) {
    if (sh >= 0) return w << sh;
    if (sh < -63) return 0;
    return ((w >> (-sh - 1)) + 1) >> 1;
}

// Balanced base-256 digits of row g of an 8-row tile over one block (the FP64 values
// x[0 .. 2 kEB - 1] held by the four lanes t of the row: columns 8 j + 2t and 8 j + 2t + 1 in
// x[2j], x[2j + 1]), written as bf16 pairs to F[kh] (the tile's slices of the block's columns
// 16 kh .. 16 kh + 15) in the tensor cores' K-major layout: [slice][core matrix of 8 columns]
// [row][8 bf16], 16 bytes per row and 128 per core matrix; and the row scale 2^(em - 1021) to
// *scale (lane t = 0).  The digit scheme is described at factor_emulated.
__device__ __forceinline__ void slice_row(const double (&x)[2 * kEB], uint32_t* F0, uint32_t* F1, double* scale) {
    const int lane = threadIdx.x & 31;
    int em = 0;
#pragma unroll
    for (int i = 0; i < 2 * kEB; ++i) em = max(em, (int)((__double_as_longlong(x[i]) >> 52) & 0x7FF));
    em = max(em, __shfl_xor_sync(0xffffffffu, em, 1));
    em = max(em, __shfl_xor_sync(0xffffffffu, em, 2));
#pragma unroll
    for (int kk = 0; kk < kEK; ++kk) {
        uint32_t* F = kk ? F1 : F0;
        unsigned long long Yb[4];
        bool negx[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {  // columns 16 kk + {2t, 2t + 1, 8 + 2t, 8 + 2t + 1}
            const unsigned long long bits = (unsigned long long)__double_as_longlong(x[4 * kk + i]);
            const int E = (int)((bits >> 52) & 0x7FF);
            unsigned long long Y = 0;  // |x| 2^(1077 - em) rounded to nearest, below 2^55
            if (E > 0 && E < 0x7FF) {  // zero and subnormals slice to zero
                const int sh = em - E;
                const unsigned long long M = ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2;
                Y = sh == 0 ? M : sh >= 56 ? 0ull : ((M >> (sh - 1)) + 1) >> 1;
            }
            // adding 128 to each of the six lower digits lets every digit be read as a byte
            // minus 128; the top digit keeps the rest (0 .. 128)
            Yb[i] = Y + 0x808080808080ull;
            negx[i] = (bits >> 63) != 0;
        }
#pragma unroll
        for (int ss = 0; ss < 7; ++ss) {  // ss = 0: the most significant digit
            uint32_t h16[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int qv = ss == 0 ? (int)(Yb[i] >> 48) : (int)((Yb[i] >> (48 - 8 * ss)) & 255ull) - 128;
                if (negx[i]) qv = -qv;
                h16[i] = __float_as_uint((float)qv) >> 16;  // exact: |qv| <= 2^7
            }
            // lane = 4 g + t: row g, columns 2t, 2t + 1 of the core matrices of columns 0-7 and 8-15
            F[ss * 64 + lane] = h16[0] | (h16[1] << 16);
            F[ss * 64 + 32 + lane] = h16[2] | (h16[3] << 16);
        }
    }
    if ((lane & 3) == 0) *scale = em > 0 ? __longlong_as_double((long long)(em + 2) << 52) : 0.0;
}

// Row tile it below the factorised diagonal block of tile columns K0 .. K0 + kEB - 1 (inverses
// of its diagonal tiles in Tblk): L_it,K0+j = (A_it,K0+j - sum_{k<j} L_it,K0+k L_K0+j,K0+k^T)
// Ti_j^T for j < kEB on the FP64 tensor path, one warp, the row's tiles in registers.  The warp's
// scratch tile W turns each result from the accumulator into the operand layout.  The
// results are stored to A and sliced for the trailing update (F, scale: this tile's slices
// and row scales).
__device__ void block_rows(double* A, int it, int K0, const double* Tblk, double* W, uint32_t* F0, uint32_t* F1,
                           double* scale) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    double* R = A + tix(it, K0);  // tiles (it, K0 .. K0 + kEB - 1), contiguous
    double x[2 * kEB];            // accumulator layout: tile j holds columns 2t, 2t + 1 of row g
#pragma unroll
    for (int j = 0; j < kEB; ++j) {
        x[2 * j] = R[64 * j + te(g, 2 * t)];
        x[2 * j + 1] = R[64 * j + te(g, 2 * t + 1)];
    }
    double xa[kEB - 1][2];  // operand layout of the solved tiles: columns t and 4 + t of row g
#pragma unroll
    for (int j = 0; j < kEB; ++j) {
        double a0 = x[2 * j], a1 = x[2 * j + 1];
        const double* Lj = A + tix(K0 + j, K0);  // tiles (K0 + j, K0 .. K0 + j), contiguous
#pragma unroll
        for (int k = 0; k < j; ++k) {
            dmma(a0, a1, neg(xa[k][0]), Lj[64 * k + te(g, t)]);
            dmma(a0, a1, neg(xa[k][1]), Lj[64 * k + te(g, 4 + t)]);
        }
        W[te(g, 2 * t)] = a0;
        W[te(g, 2 * t + 1)] = a1;
        __syncwarp();
        const double p0 = W[te(g, t)], p1 = W[te(g, 4 + t)];
        __syncwarp();
        const double* Ti = Tblk + 64 * j;
        double y0 = 0.0, y1 = 0.0;
        dmma(y0, y1, p0, Ti[te(g, t)]);
        dmma(y0, y1, p1, Ti[te(g, 4 + t)]);
        R[64 * j + te(g, 2 * t)] = y0;
        R[64 * j + te(g, 2 * t + 1)] = y1;
        x[2 * j] = y0;
        x[2 * j + 1] = y1;
        if (j < kEB - 1) {
            W[te(g, 2 * t)] = y0;
            W[te(g, 2 * t + 1)] = y1;
            __syncwarp();
            xa[j][0] = W[te(g, t)];
            xa[j][1] = W[te(g, 4 + t)];
            __syncwarp();
        }
    }
    slice_row(x, F0, F1, scale + g);
}

// Per-CTA workspace of the emulated factorisation: for each of the block's two 16-column halves
// the slices of the rows below the current block ([row tile][7 slices][2 core matrices], 1792
// bytes per row tile), npad row scales, then the inverses of all diagonal tiles ([npad / 8][64]
// doubles).
__device__ __forceinline__ unsigned char* emu_ws(const SolveCtx& c) { return c.ws_e + (int64_t)blockIdx.x * c.ws_e_stride; }
__device__ __forceinline__ int64_t emu_half_bytes(int npad) { return (int64_t)(npad / 8) * kSliceTileBytes; }
__device__ __forceinline__ int emu_rows(const SolveCtx& c) { return c.nrow > 0 ? c.nrow : c.npad; }
__device__ __forceinline__ double* emu_tile_inverses(const SolveCtx& c) {
    return reinterpret_cast<double*>(emu_ws(c) + 2 * emu_half_bytes(emu_rows(c))) + emu_rows(c);
}

// ---- tensor-core (tcgen05) helpers for the emulated updates --------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16 bytes,
// the next along K lbo bytes on, the next along M or N sbo bytes on.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D, M = 128, N = 8 kColT.
constexpr uint32_t kUmmaIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(8 * kColT / 8) << 17) |
                                ((uint32_t)(128 / 16) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(kUmmaIdesc), "r"(accumulate));
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Wait for the completion of phase `parity` of an mbarrier, at most kWaitLimit polls; the
// result is the same on every thread of the CTA (false: the wait gave up somewhere).
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < kWaitLimit && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return __syncthreads_and((int)done) != 0;
}

// Tensor memory and barriers of an emulated CTA.
struct EmuTc {
    uint32_t tmem;       // base of kEmuTmemCols columns: slice group g at columns 8 kColT g
    uint32_t bar_ld;     // completion of the staging copies
    uint32_t bar_mma;    // completion of the MMAs
    uint32_t ph_ld, ph_mma;
    bool dead;           // a bounded wait gave up: take no more work
};

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// A bounded wait gave up: record it; the CTA stops taking work.
__device__ __forceinline__ bool emu_fail(const SolveCtx& c, EmuTc& tc) {
    if (threadIdx.x == 0) atomicOr(c.err, kErrTimeout);
    tc.dead = true;
    return false;
}

// Trailing update C -= P P^T of the M = Nt - K1 row tiles below the block that ends at K1, on
// the tensor cores.  P's rows are cut into seven digit slices (see factor_emulated), and every
// slice group G_g = sum_{s+t=g} P_s P_t^T is accumulated exactly in FP32 in tensor memory.
// Output tiles of kBandT row tiles (128 rows) by kColT row tiles (32 columns) cover the lower
// triangle, band by band.  Bulk copies stage the band's slices (A, both 16-column halves of the
// block) once per band and each column tile's slices (B) in one of two buffers, the next tile's
// while the current one computes.  One thread issues the 68 slice products of a tile (34 slice
// pairs x 2 halves) into the 8 group accumulators; all 8 warps then read their rows (lane
// quadrant warp % 4) and columns (half warp / 4) of the groups, pack each element's groups into
// one integer and subtract it as an FP64 value.
// With appended query rows (tiles Ntr .. Nt - 1, see fit_instance) only the diagonal tiles of
// the query-by-query block are needed: its other column tiles are skipped.
__device__ bool trailing_update_tc(const SolveCtx& c, double* A, int Nt, int Ntr, int K1, const unsigned char* E,
                                   int64_t KH, const double* sr, unsigned char* stage, EmuTc& tc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int M = Nt - K1;
    const int jr = (max(Ntr - K1, 0) + kColT - 1) / kColT;  // column tiles of the matrix itself
    const int next1 = min(K1 + kEB, Ntr);                     // end of the next block's columns
    const uint32_t aA = smem_addr(stage), aB = aA + kStageA;
    const int q = warp & 3, h = warp >> 2;  // lane quadrant (rows 32 q ..) and column half
    const int row = 32 * q + lane, rb = row >> 3, rr = row & 7;
    for (int b0 = 0; b0 < M; b0 += kBandT) {
        const int nb = min(kBandT, M - b0);
        const bool rvalid = rb < nb;
        const int rt = K1 + b0 + rb;
        const int er = rvalid ? (int)(__double_as_longlong(sr[8 * (b0 + rb) + rr]) >> 52) : 0;
        const int n_tiles = (b0 + nb + kColT - 1) / kColT;  // column tiles reaching the band's last row tile
        // column tiles of appended query rows: only those that meet the band's rows
        const int qstart = max(jr, b0 / kColT);
        auto next_tile = [&](int j) { return j + 1 < jr ? j + 1 : max(j + 1, qstart); };
        const int first = jr > 0 ? 0 : qstart;
        if (first >= n_tiles) continue;
        if (tid == 0) {  // the band's A and the first column tile's B (buffer 0)
            const int nc = min(kColT, M - first * kColT);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc.bar_ld),
                         "r"((uint32_t)(2 * (nb + nc) * kSliceTileBytes))
                         : "memory");
            for (int kh = 0; kh < 2; ++kh) {
                const unsigned char* H = E + kh * KH;
                bulk_load(stage + kh * kBandT * kSliceTileBytes, H + (int64_t)b0 * kSliceTileBytes,
                          (uint32_t)nb * kSliceTileBytes, tc.bar_ld);
                bulk_load(stage + kStageA + kh * kColT * kSliceTileBytes, H + (int64_t)first * kColT * kSliceTileBytes,
                          (uint32_t)nc * kSliceTileBytes, tc.bar_ld);
            }
        }
        for (int jt = first, kb = 0; jt < n_tiles; jt = next_tile(jt), ++kb) {
            const int c0 = jt * kColT, nc = min(kColT, M - c0);
            const uint32_t bufB = aB + (uint32_t)((kb & 1) * kStageB);
            if (!bar_wait(tc.bar_ld, tc.ph_ld)) return emu_fail(c, tc);
            tc.ph_ld ^= 1;
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int kh = 0; kh < 2; ++kh)
#pragma unroll
                    for (int ss = 0; ss < 7; ++ss)
#pragma unroll
                        for (int tt = 0; tt < 7 && ss + tt < 8; ++tt) {
                            const int gq = ss + tt;
                            umma_bf16(tc.tmem + gq * 8 * kColT,
                                      umma_desc(aA + kh * kBandT * kSliceTileBytes + ss * 256, 128, kSliceTileBytes),
                                      umma_desc(bufB + kh * kColT * kSliceTileBytes + tt * 256, 128, kSliceTileBytes),
                                      // the first product of a group (pair (0, g), or (1, 6)
                                      // for g = 7) overwrites the accumulator
                                      (kh == 0 && (ss == 0 || (ss == 1 && gq == 7))) ? 0u : 1u);
                        }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc.bar_mma)
                             : "memory");
                if (next_tile(jt) < n_tiles) {  // the next column tile's B into the other buffer
                    const int c1 = next_tile(jt) * kColT, n1 = min(kColT, M - c1);
                    unsigned char* dst = stage + kStageA + ((kb + 1) & 1) * kStageB;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc.bar_ld),
                                 "r"((uint32_t)(2 * n1 * kSliceTileBytes))
                                 : "memory");
                    for (int kh = 0; kh < 2; ++kh)
                        bulk_load(dst + kh * kColT * kSliceTileBytes, E + kh * KH + (int64_t)c1 * kSliceTileBytes,
                                  (uint32_t)n1 * kSliceTileBytes, tc.bar_ld);
                }
            }
            // while the MMAs run: this thread's 16 entries of C (row `row`, the 8 columns of each
            // of its two column tiles) and the column scales, all loads issued at once
            long long cv[2][8];
            int ec[2][8];
            bool ok[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int cb = 2 * h + j, ct = K1 + c0 + cb;
                ok[j] = rvalid && cb < nc && ct <= rt && (ct < Ntr || ct == rt);
                const double* C = A + tix(ok[j] ? rt : K1, ok[j] ? ct : K1);
                const double* scl = sr + 8 * (ok[j] ? c0 + cb : 0);
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    cv[j][cc] = ok[j] ? __double_as_longlong(C[te(rr, cc)]) : 0;
                    ec[j][cc] = (int)(__double_as_longlong(scl[cc]) >> 52);
                }
            }
            if (!bar_wait(tc.bar_mma, tc.ph_mma)) return emu_fail(c, tc);
            tc.ph_mma ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // the thread's two column tiles of the output tile
                const int cb = 2 * h + j;
                // a warp none of whose rows is updated in this column tile (rows past the band,
                // above the diagonal, or of the query block away from its diagonal) skips it;
                // the test is warp-uniform, as the collective tcgen05.ld needs
                if (!__any_sync(0xffffffffu, ok[j])) continue;
#pragma unroll
                for (int p = 0; p < 2; ++p) {  // four columns at a time
                    uint32_t v[8][4];
#pragma unroll
                    for (int gq = 0; gq < 8; ++gq)
                        tmem_ld4(tc.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(gq * 8 * kColT + 8 * cb + 4 * p), v[gq]);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int cc = 4 * p + e;
                        // each group read from the bits of G + 1.5 * 2^23 (exact: |G| < 2^22)
                        long long gq8[8];
#pragma unroll
                        for (int gq = 0; gq < 8; ++gq) gq8[gq] = __float_as_int(__uint_as_float(v[gq][e]) + 12582912.0f);
                        constexpr long long kOffBits = 0x4B400000ll * 0x01010101ll;
                        const long long hi = gq8[0] * (1ll << 24) + gq8[1] * (1ll << 16) + gq8[2] * 256 + gq8[3] - kOffBits;
                        const long long lo = gq8[4] * (1ll << 24) + gq8[5] * (1ll << 16) + gq8[6] * 256 + gq8[7] - kOffBits;
                        // the update is w 2^(er + ec - 2102), in units of 2^-kFixBits
                        cv[j][cc] -= fix_shift(hi * (1ll << 16) + ((lo + (1ll << 15)) >> 16),
                                               er + ec[j][cc] - (2102 - kFixBits));
                    }
                }
            }
            // the next block's columns are final after this update: stored as FP64 (see
            // factor_emulated), the rest in the fixed point
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (ok[j]) {
                    const int ct = K1 + c0 + 2 * h + j;
                    double* C = A + tix(rt, ct);
                    if (ct < next1) {
#pragma unroll
                        for (int cc = 0; cc < 8; ++cc) C[te(rr, cc)] = double_of_fix(cv[j][cc]);
                    } else {
#pragma unroll
                        for (int cc = 0; cc < 8; ++cc) C[te(rr, cc)] = __longlong_as_double(cv[j][cc]);
                    }
                }
            // every thread's reads of the accumulators are done before the next tile's MMAs
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    return true;
}

// Right-looking Cholesky of a global-memory instance in blocks of W = 8 kEB columns, with
// every trailing update C -= P P^T (P: the block's W columns below it) done on the bf16
// tensor cores to FP64 accuracy.  Each row r of P is written exactly as
//     P_r = 2^(e_r - 1021) sum_{s=1..7} q_rs 2^(-8 s),   q_rs integer, |q_rs| <= 128,
// from the bits of its FP64 values aligned to the row's largest biased exponent e_r (rounded
// to nearest at 2^-55 of the row maximum): a 55-bit integer per value, cut into seven
// balanced base-256 digits (the lower six in [-128, 127], the top one in [0, 128]), each
// exact in bf16.  A slice product Q_s Q_t^T sums W <= 64 products of at most 2^14, so every
// group G_g = sum_{s+t=g} Q_s Q_t^T with g <= 9 (at most 7 terms) is an integer below 2^23
// and accumulates exactly in FP32; groups g >= 10 are below 2^-64 relative and dropped.  The
// FP64 update is
//     C_rc -= 2^(e_r + e_c - 2042) sum_g 2^(-8 g) G_g,rc.
// The groups are packed exactly into two 64-bit integers, hi (g = 2..5) and lo (g = 6..9),
// and joined as w = 2^16 hi + round(lo / 2^16), below 2^63 because every group stays below
// 2^22 with W = 32: the rounding of lo is below 2^-57 of the scale 2^(e_r + e_c - 2042).  The
// trailing matrix is held in the fixed point of kFixBits (assembled so by fit_instance): w is
// shifted to it and subtracted as an integer, so an updated entry costs no FP64 operation,
// and each block's columns are stored as FP64 by the update that completes them.  The slice
// products run on the tensor cores
// (trailing_update_tc); within a block the diagonal block is factorised as in the plain loop
// (8x8 tiles, FP64 tensor path) and the rows below it are solved one row tile per warp
// (block_rows), which also writes their slices.
// Nt row tiles, of which the first Ntr are factorised (Nt > Ntr: appended query rows, whose
// rows below are solved and whose diagonal tiles are updated, but not factorised).
__device__ bool factor_emulated(const SolveCtx& c, const Shared& s, double* A, int Nt, int Ntr, int* s_fail,
                                EmuTc& tc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    unsigned char* E = emu_ws(c);
    const int64_t KH = emu_half_bytes(emu_rows(c));
    double* sr = reinterpret_cast<double*>(E + 2 * KH);  // row scales of the rows below the block
    double* Tall = emu_tile_inverses(c);                  // inverses of all diagonal tiles, for the solves
    for (int K0 = 0; K0 < Ntr; K0 += kEB) {
        const int K1 = min(K0 + kEB, Ntr);
        // the first block's columns (tiles (it, jt), jt < K1, jt <= it) from the fixed point of
        // the assembly to FP64; later blocks' columns are stored as FP64 by the trailing update
        // that completes them
        if (K0 == 0) {
            const int nb = K1 - K0;
            const int64_t ne = (int64_t)(Nt - K0) * nb * 64;
            for (int64_t x = tid; x < ne; x += blockDim.x) {
                const int p = (int)(x >> 6), it = K0 + p / nb, jt = K0 + p % nb;
                if (jt > it) continue;
                double* v = A + tix(it, jt) + (x & 63);
                *v = double_of_fix(__double_as_longlong(*v));
            }
            __syncthreads();
        }
        // the diagonal block: tiles (it, jt), K0 <= jt <= it < K1, right-looking by 8 columns
        for (int kt = K0; kt < K1; ++kt) {
            double* Ti = s.Tblk + 64 * (kt - K0);
            if (warp == 0) {
                if (diag_tile_warp(A, kt, s, Ti, s.Wsc)) {
                    Tall[64 * kt + lane] = Ti[lane];
                    Tall[64 * kt + lane + 32] = Ti[lane + 32];
                } else if (lane == 0) {
                    *s_fail = 1;
                }
            }
            __syncthreads();
            if (*s_fail) return false;
            panel_column(A, kt, K1, Ti);
            __syncthreads();
            const int nj = K1 - kt - 1;
            for (int p = warp; p < nj * (nj + 1) / 2; p += nwarps) {
                const int ir = tri_row(p), it = kt + 1 + ir, jt = kt + 1 + (p - ir * (ir + 1) / 2);
                double* C = A + tix(it, jt);
                const double* Li = A + tix(it, kt);
                const double* Lj = A + tix(jt, kt);
                double c0 = C[te(g, 2 * t)], c1 = C[te(g, 2 * t + 1)];
                dmma(c0, c1, neg(Li[te(g, t)]), Lj[te(g, t)]);
                dmma(c0, c1, neg(Li[te(g, 4 + t)]), Lj[te(g, 4 + t)]);
                C[te(g, 2 * t)] = c0;
                C[te(g, 2 * t + 1)] = c1;
            }
            __syncthreads();
        }
        if (K1 >= Nt) break;
        // the rows below: one warp per row tile solves its four tiles against the diagonal
        // block and writes their slices (both column halves) and row scales
        for (int it = K1 + warp; it < Nt; it += nwarps)
            block_rows(A, it, K0, s.Tblk, s.Wsc + 64 * warp,
                       reinterpret_cast<uint32_t*>(E + (int64_t)(it - K1) * kSliceTileBytes),
                       reinterpret_cast<uint32_t*>(E + KH + (int64_t)(it - K1) * kSliceTileBytes), sr + 8 * (it - K1));
        // the slices are read by the copy engine (async proxy)
        asm volatile("fence.proxy.async;" ::: "memory");
        __syncthreads();
        if (!trailing_update_tc(c, A, Nt, Ntr, K1, E, KH, sr, s.stage, tc)) return false;
    }
    return true;
}

// Assemble A, factorise, solve alpha.  Returns false if a pivot was not positive.
// Local coordinates of the query at position p (id qid) of instance I (defined below).
__device__ __forceinline__ void query_local(const SolveCtx& c, int I, int64_t p, int64_t qid, double xl[3],
                                            int* qi = nullptr);

// Latent variance by bordering (emulated kernel, nq > 0 queries of instance I from position q0):
// the matrix is padded to Nr = 32 ceil(N / 32) rows and the kernel vectors k_a of the queries are
// appended as rows Nr + a, with k(x*, x*) = 1 on the diagonal.  Factorising only the first Nr
// columns turns row Nr + a into v_a = L^-1 k_a and leaves the Schur complement, whose diagonal
// entry is 1 - |v_a|^2 = u_a (Eq. 2).  Each appended row's arithmetic involves only that row and
// the instance's own rows, so u_a does not depend on the other queries.
template <bool kProps, bool kEmu = false>
__device__ bool fit_instance(const SolveCtx& c, const Shared& s, int N, int64_t base, EmuTc* tc = nullptr, int nq = 0,
                             int64_t q0 = 0, int I = 0) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    const int g = lane >> 2, t = lane & 3;
    __shared__ int s_fail;
    const int Np = nq > 0 ? (N + 31) & ~31 : (N + 7) & ~7, Nt = Np >> 3;  // the instance's rows (Nr)
    const int Ntq = Nt + (nq + 7) / 8;                                   // with the appended rows
    const bool lattice = c.b.Xi != nullptr;
    for (int e = tid; e < 3 * N; e += nt) {
        double v = c.b.Xl[3 * base + e];
        s.X[e] = v;
        s.Xf[e] = (float)v;
        // the point's own FP32 world coordinate, recovered exactly (the FP64 local value
        // differs from it by the centre up to a rounding far below half an FP32 ulp)
        if (kEmu && !lattice) s.Xw[e] = (float)(v + (c.b.centre ? c.b.centre[3 * (int64_t)I + e % 3] : 0.0));
    }
    if (lattice)
        for (int e = tid; e < N; e += nt) {
            const char4 q = c.b.Xi[base + e];
            s.xi[e] = ((int)q.x + 16) | (((int)q.y + 16) << 8) | (((int)q.z + 16) << 16);
        }
    if (nq > 0)  // local coordinates of the appended queries (NaN: not finite, row left zero)
        for (int a = tid; a < nq; a += nt) {
            const int64_t p = q0 + a;
            const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
            double xl[3];
            int qi = 0;
            query_local(c, I, p, qid, xl, &qi);
            const bool fin = isfinite(xl[0]) && isfinite(xl[1]) && isfinite(xl[2]);
            if (lattice) {  // the lattice code (its bits: a tiny float, never NaN); [1]: finite flag
                s.qw[3 * a] = __int_as_float(qi);
                s.qw[3 * a + 1] = fin ? 0.f : NAN;
            } else {
                for (int k = 0; k < 3; ++k)
                    s.qw[3 * a + k] = fin ? (float)(xl[k] + (c.b.centre ? c.b.centre[3 * (int64_t)I + k] : 0.0)) : NAN;
            }
        }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    double* A = s.A;
    // A = K + sigma^2 I in 8x8 tiles (Sec. III-A kernel, Eq. 1 noise term); padding rows and
    // columns are the identity so the padded factor is block-diagonal.  The emulated kernel
    // writes the fixed point of kfix_pair (appended query rows: the query's kernel values, 1
    // on the diagonal, and only the diagonal tiles of the query-by-query block).
    const int64_t ntl = n_tiles(Ntq);
    if (kEmu)
        for (int64_t tl = warp; tl < ntl; tl += nwarps) {
            const int it = tri_row((int)tl), jt = (int)tl - it * (it + 1) / 2;
            if (jt >= Nt && jt != it) continue;
            for (int e = lane; e < 64; e += 32) {
                const int i = 8 * it + (e >> 3), j = 8 * jt + (e & 7);
                long long v;
                if (i >= Np) {  // appended query row a = i - Np
                    const int a = i - Np;
                    if (j >= Np || a >= nq) {
                        v = (i == j) ? (1ll << kFixBits) : 0;
                    } else if (j >= N || isnan(s.qw[3 * a + 1])) {
                        v = 0;
                    } else if (lattice) {
                        v = fix_of_double(c.P.lat_tab[lat_m(s.xi[j], __float_as_int(s.qw[3 * a]))]);
                    } else if (c.P.precision == VGP_MIXED) {
                        v = kfix_ff(s.qw + 3 * a, s.Xw + 3 * j, c.P.inv2l2_hi, c.P.inv2l2_lo, s.Tff);
                    } else {
                        // the query's FP64 local coordinates, formed as query_local forms them
                        double r2 = 0.0;
                        for (int k = 0; k < 3; ++k) {
                            const double cen = c.b.centre ? c.b.centre[3 * (int64_t)I + k] : 0.0;
                            const double d = s.X[3 * j + k] - ((double)s.qw[3 * a + k] - cen);
                            r2 += d * d;
                        }
                        v = fix_of_double(exp(-r2 * c.P.inv2l2));
                    }
                } else if (i >= N || j >= N) v = (i == j) ? (1ll << kFixBits) : 0;
                else if (j > i) v = 0;
                else if (j == i) v = fix_of_double(1.0 + c.P.s2);  // s2: sigma_prop^2 for properties
                else v = kfix_pair(c.P, s, lattice, i, j);
                A[tl * 64 + te(e >> 3, e & 7)] = __longlong_as_double(v);
            }
        }
    else
    for (int64_t tl = warp; tl < ntl; tl += nwarps) {
        const int it = tri_row((int)tl), jt = (int)tl - it * (it + 1) / 2;
        if (jt >= Nt && jt != it) continue;
        for (int e = lane; e < 64; e += 32) {
            const int i = 8 * it + (e >> 3), j = 8 * jt + (e & 7);
            double v;
            if (i >= N || j >= N) v = (i == j) ? 1.0 : 0.0;  // (no appended rows here)
            else if (j > i) v = 0.0;
            else if (j == i) v = 1.0 + c.P.s2;
            else v = kval_pair(c.P, s, lattice, i, j);
            A[tl * 64 + te(e >> 3, e & 7)] = v;
        }
    }
    __syncthreads();
    if (kEmu) {
        if (!factor_emulated(c, s, A, Ntq, Nt, &s_fail, *tc)) return false;
        // the staging of the tensor-core updates overwrote X, Xf and xi: reload them
        for (int e = tid; e < 3 * N; e += nt) {
            double v = c.b.Xl[3 * base + e];
            s.X[e] = v;
            s.Xf[e] = (float)v;
        }
        if (lattice)
            for (int e = tid; e < N; e += nt) {
                const char4 q = c.b.Xi[base + e];
                s.xi[e] = ((int)q.x + 16) | (((int)q.y + 16) << 8) | (((int)q.z + 16) << 16);
            }
        __syncthreads();
    } else
    for (int kt = 0; kt < Nt; ++kt) {
        // diagonal tile: 8x8 Cholesky and the inverse of its factor (FP64 pipe)
        if (tid == 0) {
            double* D = A + tix(kt, kt);
            double* W = s.Tinv;
            bool bad = false;
            for (int j = 0; j < 8 && !bad; ++j) {
                double v = D[te(j, j)];
                for (int k = 0; k < j; ++k) v -= D[te(j, k)] * D[te(j, k)];
                if (!(v > 0.0)) {
                    bad = true;
                    break;
                }
                const double d = sqrt(v), inv = 1.0 / d;
                D[te(j, j)] = d;
                s.invd[8 * kt + j] = inv;
                for (int i = j + 1; i < 8; ++i) {
                    double u = D[te(i, j)];
                    for (int k = 0; k < j; ++k) u -= D[te(i, k)] * D[te(j, k)];
                    D[te(i, j)] = u * inv;
                }
            }
            if (bad) {
                s_fail = 1;
            } else {
                for (int j = 0; j < 8; ++j) {
                    for (int i = 0; i < j; ++i) W[te(i, j)] = 0.0;
                    W[te(j, j)] = s.invd[8 * kt + j];
                    for (int i = j + 1; i < 8; ++i) {
                        double u = 0.0;
                        for (int k = j; k < i; ++k) u += D[te(i, k)] * W[te(k, j)];
                        W[te(i, j)] = -u * s.invd[8 * kt + i];
                    }
                }
            }
        }
        __syncthreads();
        if (s_fail) break;
        // panel: L_it,kt = A_it,kt * Tinv^T (kept in shared memory too when A is global)
        for (int it = kt + 1 + warp; it < Nt; it += nwarps) {
            double* T = A + tix(it, kt);
            const double a0 = T[te(g, t)], a1 = T[te(g, 4 + t)];
            const double b0 = s.Tinv[te(g, t)], b1 = s.Tinv[te(g, 4 + t)];
            double c0 = 0.0, c1 = 0.0;
            dmma(c0, c1, a0, b0);
            dmma(c0, c1, a1, b1);
            __syncwarp();
            T[te(g, 2 * t)] = c0;
            T[te(g, 2 * t + 1)] = c1;
            if (s.panel) {
                double* Pt = s.panel + (it - kt - 1) * 64;
                Pt[te(g, 2 * t)] = c0;
                Pt[te(g, 2 * t + 1)] = c1;
            }
        }
        __syncthreads();
        // trailing update A_it,jt -= L_it,kt L_jt,kt^T (kt < jt <= it) in 2x2 blocks of tiles:
        // four independent accumulators per warp, fragments from shared memory
        const int M = Nt - kt - 1;
        const int MB = (M + 1) >> 1;
        const int NB = MB * (MB + 1) / 2;
        for (int p = warp; p < NB; p += nwarps) {
            const int bi = tri_row(p), bj = p - bi * (bi + 1) / 2;
            const int i0 = 2 * bi, j0 = 2 * bj;
            double na[2][2], bb[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int ii = i0 + r, jj = j0 + r;
                const double* Pi = s.panel ? s.panel + ii * 64 : A + tix(kt + 1 + ii, kt);
                const double* Pj = s.panel ? s.panel + jj * 64 : A + tix(kt + 1 + jj, kt);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    na[r][k] = ii < M ? neg(Pi[te(g, 4 * k + t)]) : 0.0;
                    bb[r][k] = jj < M ? Pj[te(g, 4 * k + t)] : 0.0;
                }
            }
            double cc[2][2][2];
            bool valid[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int ii = i0 + r, jj = j0 + q;
                    valid[r][q] = ii < M && jj <= ii;
                    cc[r][q][0] = cc[r][q][1] = 0.0;
                    if (valid[r][q]) {
                        const double* C = A + tix(kt + 1 + ii, kt + 1 + jj);
                        cc[r][q][0] = C[te(g, 2 * t)];
                        cc[r][q][1] = C[te(g, 2 * t + 1)];
                    }
                }
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int q = 0; q < 2; ++q) dmma(cc[r][q][0], cc[r][q][1], na[r][k], bb[q][k]);
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (valid[r][q]) {
                        double* C = A + tix(kt + 1 + i0 + r, kt + 1 + j0 + q);
                        C[te(g, 2 * t)] = cc[r][q][0];
                        C[te(g, 2 * t + 1)] = cc[r][q][1];
                    }
        }
        __syncthreads();
    }
    if (s_fail) return false;
    // The solves use the instance's own 8-row tiles only: the leading block of the factor is the
    // factor of the leading block, so rows padded to 32 for appended queries change no bit of
    // alpha (the solves' work split depends on the tile count).
    const int Ns = (N + 7) & ~7, Nts = Ns >> 3;
    if (kProps) {
        // property weights alpha_c = A^-1 y_c, one right-hand side per channel (Eq. 6)
        for (int ch = 0; ch < c.b.nprop; ++ch) {
            for (int i = tid; i < Ns; i += nt) s.z[i] = i < N ? c.b.yprop[(base + i) * c.b.nprop + ch] : 0.0;
            __syncthreads();
            if (kEmu)
                chol_solve_inv(s, A, Nts, s.pa[ch], emu_tile_inverses(c));
            else
                chol_solve(s, A, Nts, s.pa[ch]);
        }
        return true;
    }
    // alpha = A^-1 1 (Eq. 1)
    for (int i = tid; i < Ns; i += nt) s.z[i] = i < N ? 1.0 : 0.0;
    __syncthreads();
    if (kEmu)
        chol_solve_inv(s, A, Nts, s.alpha, emu_tile_inverses(c));
    else
        chol_solve(s, A, Nts, s.alpha);
    for (int j = tid; j < Ns; j += nt) {
        const float hi = (float)s.alpha[j];
        s.alf[j] = hi;
        s.alf_lo[j] = (float)(s.alpha[j] - (double)hi);
    }
    __syncthreads();
    return true;
}

struct EvalOut {
    double d, g[3], v;
    int status;
};

// Reverting (Eq. 3), distance variance (Eq. 4), chain-rule gradient, with the caps of the
// occupancy: lo = log o, gro = grad o / o.
__device__ __forceinline__ void revert(const DevParams& P, double lo, const double gro[3], double u, bool want_var,
                                       EvalOut& r) {
    if (!(lo >= P.log_floor)) {  // also catches NaN (o <= 0)
        r.status = VGP_ST_CLAMPED;
        r.d = P.d_max;
        r.g[0] = r.g[1] = r.g[2] = 0.0;
        r.v = INFINITY;
        return;
    }
    r.status = VGP_ST_OK;
    if (lo >= 0.0) {
        const double lam = -P.l2 / P.d_var_floor;
        r.d = 0.0;
        r.g[0] = r.g[1] = r.g[2] = 0.0;
        r.v = want_var ? lam * lam * u : NAN;
        return;
    }
    const double d = sqrt(-2.0 * P.l2 * lo);
    r.d = d;
    for (int a = 0; a < 3; ++a) r.g[a] = -P.l2 * gro[a] / d;
    if (want_var) {
        const double o = exp(lo);
        const double lam = -P.l2 / (o * fmax(d, P.d_var_floor));
        r.v = lam * lam * u;
    } else {
        r.v = NAN;
    }
}

__device__ __forceinline__ void write_out(const SolveBatch& b, int64_t qid, const EvalOut& r) {
    b.d[qid] = r.d;
    if (b.grad) {
        b.grad[3 * qid] = r.g[0];
        b.grad[3 * qid + 1] = r.g[1];
        b.grad[3 * qid + 2] = r.g[2];
    }
    if (b.var) b.var[qid] = r.v;
    if (b.status) b.status[qid] = (uint8_t)r.status;
}

__device__ __forceinline__ void query_local(const SolveCtx& c, int I, int64_t p, int64_t qid, double xl[3],
                                            int* qi) {
    double xg[3];
    if (c.b.qkey) {
        int i, j, k;
        unpack_key(c.b.qkey[p], i, j, k);
        if (qi && c.b.inst_key) {
            int lx, ly, lz;
            unpack_key(c.b.inst_key[I], lx, ly, lz);
            // offsets relative to the instance leaf origin, biased by 16 into 0..255
            *qi = (i - 8 * lx + 16) | ((j - 8 * ly + 16) << 8) | ((k - 8 * lz + 16) << 16);
        }
        xg[0] = (double)i * c.P.vs;
        xg[1] = (double)j * c.P.vs;
        xg[2] = (double)k * c.P.vs;
    } else {
        const int64_t qp = qid / c.b.qdiv;
        xg[0] = (double)c.b.qxyz[3 * qp];
        xg[1] = (double)c.b.qxyz[3 * qp + 1];
        xg[2] = (double)c.b.qxyz[3 * qp + 2];
    }
    for (int a = 0; a < 3; ++a) xl[a] = xg[a] - c.b.centre[3 * (int64_t)I + a];
}

// Latent mean and gradient at one query; returns lo = log o and gro = grad o / o.
// qi: biased lattice offsets of the query (lattice instances only).
__device__ __forceinline__ void latent_mean(const DevParams& P, const Shared& s, int N, bool lattice, int qi,
                                            const double xl[3], double& lo, double gro[3]) {
    if (P.precision == VGP_MIXED) {
        // FP32 kernel values and FP32 accumulation.  Off the lattice, the nearest training point
        // shifts the exponent (exp(-(r^2 - r0^2) / 2l^2) <= 1, no underflow).  The sum is
        // compensated: alpha is carried as two floats and the rounding error of every product
        // and addition is accumulated separately (Neumaier), all on the FP32 pipe.
        const float qx = (float)xl[0], qy = (float)xl[1], qz = (float)xl[2];
        float r0 = 0.f;
        if (!lattice) {
            r0 = INFINITY;
            for (int j = 0; j < N; ++j) {
                float dx = s.Xf[3 * j] - qx, dy = s.Xf[3 * j + 1] - qy, dz = s.Xf[3 * j + 2] - qz;
                r0 = fminf(r0, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            }
        }
        float sum = 0.f, comp = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int j = 0; j < N; ++j) {
            float dx = s.Xf[3 * j] - qx, dy = s.Xf[3 * j + 1] - qy, dz = s.Xf[3 * j + 2] - qz;
            float e;
            if (lattice) {
                e = P.lat_tab_f[lat_m(s.xi[j], qi)];
            } else {
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                e = exp2f((r0 - r2) * P.inv2l2_log2e);
            }
            const float ah = s.alf[j];
            const float w = ah * e;
            comp += fmaf(ah, e, -w) + s.alf_lo[j] * e;
            const float t2 = sum + w;
            comp += fabsf(sum) >= fabsf(w) ? (sum - t2) + w : (w - t2) + sum;
            sum = t2;
            gx = fmaf(w, dx, gx);
            gy = fmaf(w, dy, gy);
            gz = fmaf(w, dz, gz);
        }
        const double tot = (double)sum + (double)comp;
        if (!(tot > 0.0)) {
            lo = NAN;
            gro[0] = gro[1] = gro[2] = 0.0;
            return;
        }
        lo = -(double)r0 * P.inv2l2 + log(tot);
        const double inv = 1.0 / (tot * P.l2);
        gro[0] = (double)gx * inv;
        gro[1] = (double)gy * inv;
        gro[2] = (double)gz * inv;
    } else {
        double o = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int j = 0; j < N; ++j) {
            double dx = s.X[3 * j] - xl[0], dy = s.X[3 * j + 1] - xl[1], dz = s.X[3 * j + 2] - xl[2];
            double k;
            if (lattice) k = P.lat_tab[lat_m(s.xi[j], qi)];
            else k = exp(-(dx * dx + dy * dy + dz * dz) * P.inv2l2);
            const double w = s.alpha[j] * k;
            o += w;
            gx += w * dx;
            gy += w * dy;
            gz += w * dz;
        }
        if (!(o > 0.0)) {
            lo = NAN;
            gro[0] = gro[1] = gro[2] = 0.0;
            return;
        }
        lo = log(o);
        const double inv = 1.0 / (o * P.l2);
        gro[0] = gx * inv;
        gro[1] = gy * inv;
        gro[2] = gz * inv;
    }
}

// u = 1 - |L^-1 k|^2 (Eq. 2) with FP64 kernel values; the thread's own column of V lives in
// global workspace.
__device__ __forceinline__ double latent_var(const DevParams& P, const Shared& s, int N, bool lattice, int qi,
                                             const double xl[3], double* V, int stride) {
    const double* A = s.A;
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
        double sum;
        if (lattice) {
            sum = P.lat_tab[lat_m(s.xi[i], qi)];
        } else {
            double dx = s.X[3 * i] - xl[0], dy = s.X[3 * i + 1] - xl[1], dz = s.X[3 * i + 2] - xl[2];
            const double y = -(dx * dx + dy * dy + dz * dz) * P.inv2l2;
            sum = P.precision == VGP_MIXED ? exp_neg(y, s.T256) : exp(y);
        }
        const int it = i >> 3, r = i & 7;
        for (int jt = 0; jt < it; ++jt) {
            const double* T = A + tix(it, jt);
#pragma unroll
            for (int c2 = 0; c2 < 8; ++c2) sum -= T[te(r, c2)] * V[(int64_t)(8 * jt + c2) * stride];
        }
        const double* T = A + tix(it, it);
        for (int c2 = 0; c2 < r; ++c2) sum -= T[te(r, c2)] * V[(int64_t)(8 * it + c2) * stride];
        const double vi = sum * s.invd[i];
        V[(int64_t)i * stride] = vi;
        acc += vi * vi;
    }
    return fmax(0.0, 1.0 - acc);
}

// Property means c_ch = sum_j alpha_ch,j k_j (Eq. 6) in FP64 with FP64 kernel values.
__device__ __forceinline__ void property_mean(const DevParams& P, const Shared& s, int N, int nprop,
                                              bool lattice, int qi, const double xl[3], double* out) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < N; ++j) {
        double k;
        if (lattice) {
            k = P.lat_tab[lat_m(s.xi[j], qi)];
        } else {
            double dx = s.X[3 * j] - xl[0], dy = s.X[3 * j + 1] - xl[1], dz = s.X[3 * j + 2] - xl[2];
            k = exp(-(dx * dx + dy * dy + dz * dz) * P.inv2l2);
        }
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            if (ch < nprop) acc[ch] += s.pa[ch][j] * k;
    }
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
        if (ch < nprop) out[ch] = acc[ch];
}

__device__ __forceinline__ void invalid(EvalOut& r, int status) {
    r.status = status;
    r.d = INFINITY;
    r.g[0] = r.g[1] = r.g[2] = 0.0;
    r.v = INFINITY;
}

// The body of the GP solve kernels (see k_solve below).
template <bool kProps, bool kEmu>
__device__ __forceinline__ void solve_body(const SolveCtx& c) {
    extern __shared__ __align__(128) double sm[];
    __shared__ int s_item[2];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    const int tid = threadIdx.x, nt = blockDim.x;
    double* ws_a = c.a_in_smem ? nullptr : c.ws_a + (int64_t)blockIdx.x * c.ws_a_stride;
    Shared s = carve(sm, c.npad, c.a_in_smem, ws_a, c.b.nprop, c.stage_panel, c.b.Xi != nullptr, false, kEmu);
    double* V = c.ws_v ? c.ws_v + (int64_t)blockIdx.x * c.ws_v_stride + tid : nullptr;
    const bool lattice = c.b.Xi != nullptr;
    for (int j = tid; j < 256; j += nt) s.T256[j] = c.P.exp_tab[j];
    if (kEmu)
        for (int j = tid; j < 256; j += nt) {
            float h, l;
            split_pair(c.P.exp_tab[j], h, l);
            s.Tff[j] = make_float2(h, l);
        }
    EmuTc tc{};
    if (kEmu) {
        // tensor memory for the 8 slice-group accumulators (held until the CTA exits) and the
        // barriers of the staging copies and of the MMAs
        if ((tid >> 5) == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                         "r"(kEmuTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar[0])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar[1])) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tc.tmem = s_tmem;
        tc.bar_ld = smem_addr(&s_bar[0]);
        tc.bar_mma = smem_addr(&s_bar[1]);
    }
    for (bool first = true;; first = false) {
        // the next work item: an instance, or one chunk of its queries (the instance is fitted
        // again for every chunk, so the queries of a large instance spread over the GPU).  CTA i
        // takes item i first (the CTAs of a launch are spread over the SMs in index order, so a
        // grid larger than the work stays balanced), then items from the counter.
        if (tid == 0) {
            const int w = first ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(c.counter, 1);
            // graph mode: this bucket's count and share of the order, planned on the device
            const int nb = c.plan ? c.plan[c.bucket] : c.n_work;
            const int ob = c.plan ? c.plan[5 + c.bucket] : 0;
            int k = w, ci = 0, nw = nb;
            if (c.chunk_off) {
                const int* cof = c.chunk_off + ob;  // direct launches pass the bucket's offset
                nw = cof[nb] - cof[0];
                if (w < nw) {  // the last instance whose first chunk is at or before w
                    const int t = cof[0] + w;
                    int lo = 0, hi = nb - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (cof[mid] <= t)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    k = lo;
                    ci = t - cof[lo];
                }
            }
            s_item[0] = w < nw ? (c.order ? c.order[ob + k] : c.inst_base + k) : -1;
            s_item[1] = ci;
        }
        __syncthreads();
        const int I = s_item[0], ci = s_item[1];
        __syncthreads();
        if (I < 0) break;
        const int64_t base = c.b.inst_off[I];
        const int N = (int)(c.b.inst_off[I + 1] - base);
        const int64_t qa = c.b.q_off[I], qb = c.b.q_off[I + 1];
        const int qch = c.chunk_q ? *c.chunk_q : 0;
        const int64_t q0 = qch > 0 ? min(qb, qa + (int64_t)ci * qch) : qa;
        const int64_t q1 = qch > 0 ? min(qb, q0 + qch) : qb;
        if (kProps) {
            // the variance by bordering too (see below) when the work item's queries fit the
            // appended rows: the property GP's own matrix, noise sigma_c^2
            const bool pb = kEmu && c.qmax > 0 && q1 - q0 <= c.qmax;
            const bool ok = N > 0 && fit_instance<kProps, kEmu>(c, s, N, base, &tc, pb ? (int)(q1 - q0) : 0, q0, I);
            const int Ntr = ((N + 31) & ~31) >> 3;
            // property mode: means and variance (Eq. 6, variance read as for Eq. 2)
            const int np = c.b.nprop;
            for (int64_t p = q0 + tid; p < q1; p += nt) {
                const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
                double xl[3], cm[4] = {NAN, NAN, NAN, NAN}, w = INFINITY;
                int qi = 0;
                if (ok) {
                    query_local(c, I, p, qid, xl, &qi);
                    if (isfinite(xl[0]) && isfinite(xl[1]) && isfinite(xl[2])) {
                        property_mean(c.P, s, N, np, lattice, qi, xl, cm);
                        if (pb) {
                            const int a = (int)(p - q0), ta = Ntr + (a >> 3);
                            w = fmax(0.0, double_of_fix(__double_as_longlong(s.A[tix(ta, ta) + te(a & 7, a & 7)])));
                        } else {
                            w = latent_var(c.P, s, N, lattice, qi, xl, V, nt);
                        }
                    }
                }
                for (int ch = 0; ch < np; ++ch) c.b.pc[qid * np + ch] = cm[ch];
                c.b.pw[qid] = w;
            }
            if (!ok && N > 0 && tid == 0 && !tc.dead) atomicOr(c.err, kErrFactor);
            __syncthreads();
            if (kEmu && tc.dead) break;
            continue;
        }
        // Variance by bordering (see fit_instance): the instance's queries are appended to its
        // matrix in chunks of at most qmax, one factorisation per chunk.  Every chunk repeats
        // the same arithmetic on the instance's own rows, and a query's row involves only
        // itself, so every result is independent of the chunking and of the other queries.
        const bool border = kEmu && c.b.want_var && c.qmax > 0;
        const int Ntr = ((N + 31) & ~31) >> 3;  // first appended row tile
        for (int64_t cq0 = q0;;) {
            const int64_t cq1 = border ? min(q1, cq0 + (int64_t)c.qmax) : q1;
            const bool ok = N > 0 && fit_instance<kProps, kEmu>(c, s, N, base, &tc, border ? (int)(cq1 - cq0) : 0,
                                                                 cq0, I);
            if (c.b.alpha_out && ci == 0 && cq0 == q0)
                for (int j = tid; j < N; j += nt) c.b.alpha_out[base + j] = ok ? s.alpha[j] : NAN;
            const int64_t ce = ok ? cq1 : q1;  // a failed factorisation answers all remaining queries
            for (int64_t p = cq0 + tid; p < ce; p += nt) {
                const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
                EvalOut r;
                if (!ok) {
                    invalid(r, N > 0 ? VGP_ST_FACTOR_FAIL : VGP_ST_NO_SUPPORT);
                } else {
                    double xl[3], lo, gro[3];
                    int qi = 0;
                    query_local(c, I, p, qid, xl, &qi);
                    if (!(isfinite(xl[0]) && isfinite(xl[1]) && isfinite(xl[2]))) {
                        invalid(r, VGP_ST_BAD_INPUT);
                    } else {
                        latent_mean(c.P, s, N, lattice, qi, xl, lo, gro);
                        double u = 0.0;
                        if (c.b.want_var) {
                            if (border) {  // the Schur complement's diagonal entry, clamped at 0
                                const int a = (int)(p - cq0), ta = Ntr + (a >> 3);
                                u = fmax(0.0, double_of_fix(__double_as_longlong(s.A[tix(ta, ta) + te(a & 7, a & 7)])));
                            } else {
                                u = latent_var(c.P, s, N, lattice, qi, xl, V, nt);
                            }
                        }
                        revert(c.P, lo, gro, u, c.b.want_var != 0, r);
                    }
                }
                write_out(c.b, qid, r);
            }
            if (!ok && N > 0 && tid == 0 && !tc.dead) atomicOr(c.err, kErrFactor);
            __syncthreads();
            cq0 = ce;
            if ((kEmu && tc.dead) || cq0 >= q1) break;
        }
        if (kEmu && tc.dead) break;
    }
    if (kEmu) {
        if (tc.dead) {  // let copies or MMAs still in flight finish (bounded) before releasing
            bar_wait(tc.bar_ld, tc.ph_ld);
            bar_wait(tc.bar_mma, tc.ph_mma);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if ((tid >> 5) == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc.tmem), "r"(kEmuTmemCols)
                         : "memory");
    }
}

// kProps: surface-property mode (Eq. 6); the emulated kernels run the trailing updates of
// N > 32 instances on the bf16 tensor cores (256 threads, two CTAs per SM).  Separate
// kernels, so that the plain distance kernel keeps its register budget.
template <bool kProps>
__global__ void k_solve(SolveCtx c) {
    solve_body<kProps, false>(c);
}

template <bool kProps>
__global__ void __launch_bounds__(kEmuThreads, 2) k_solve_emu(SolveCtx c) {
    solve_body<kProps, true>(c);
}

// Backward pass (derived from Eq. 1 and Eq. 3): per instance,
//   obar_q = dL/dd_q * dd/do_q, abar = sum_q obar_q k_q, lambda = A^-1 abar,
//   dL/dx_j = sum_q obar_q alpha_j k_qj (x*_q - x_j) / l^2
//             - sum_i (lambda_i alpha_j + lambda_j alpha_i) k_ij (x_i - x_j) / l^2,
// and dL/dx*_q = dL/dd_q grad d_q.  FP64 throughout; alpha is recomputed, not stored.
__global__ void k_backward(SolveCtx c) {
    extern __shared__ double sm[];
    __shared__ int s_w;
    const int tid = threadIdx.x, nt = blockDim.x;
    double* ws_a = c.a_in_smem ? nullptr : c.ws_a + (int64_t)blockIdx.x * c.ws_a_stride;
    Shared s = carve(sm, c.npad, c.a_in_smem, ws_a, 0, c.stage_panel, c.b.Xi != nullptr, true);
    const double l2 = c.P.l2;
    SolveCtx cc = c;
    cc.P.precision = VGP_FP64;
    for (int j = tid; j < 256; j += nt) s.T256[j] = c.P.exp_tab[j];
    for (;;) {
        if (tid == 0) s_w = atomicAdd(c.counter, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= c.n_work) break;
        const int I = c.order[w];
        const int64_t base = c.b.inst_off[I];
        const int N = (int)(c.b.inst_off[I + 1] - base);
        const int Nt = (N + 7) >> 3;
        const int64_t q0 = c.b.q_off[I], q1 = c.b.q_off[I + 1];
        const bool ok = N > 0 && fit_instance<false>(cc, s, N, base);
        for (int64_t p = q0 + tid; p < q1; p += nt) {
            const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
            double ob = 0.0, gq[3] = {0.0, 0.0, 0.0};
            if (ok) {
                double xl[3], lo, gro[3];
                query_local(cc, I, p, qid, xl);
                latent_mean(cc.P, s, N, false, 0, xl, lo, gro);
                EvalOut r;
                revert(cc.P, lo, gro, 0.0, false, r);
                const double gd = c.bw.dL_dd[qid];
                for (int a = 0; a < 3; ++a) gq[a] = gd * r.g[a];
                if (r.status == VGP_ST_OK && r.d > 0.0 && lo < 0.0) ob = gd * (-l2 / (exp(lo) * r.d));
            }
            c.bw.obar[p] = ob;
            if (c.bw.dL_dq)
                for (int a = 0; a < 3; ++a) c.bw.dL_dq[3 * qid + a] = gq[a];
        }
        __syncthreads();
        if (ok && c.bw.dL_dX) {
            // abar_j and the direct term, thread per training point
            for (int j = tid; j < 8 * Nt; j += nt) {
                if (j >= N) {
                    s.z[j] = 0.0;
                    continue;
                }
                double ab = 0.0, g1[3] = {0.0, 0.0, 0.0};
                for (int64_t p = q0; p < q1; ++p) {
                    const double ob = c.bw.obar[p];
                    if (ob == 0.0) continue;
                    const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
                    double xl[3];
                    query_local(cc, I, p, qid, xl);
                    double dx = xl[0] - s.X[3 * j], dy = xl[1] - s.X[3 * j + 1], dz = xl[2] - s.X[3 * j + 2];
                    double k = exp(-(dx * dx + dy * dy + dz * dz) * c.P.inv2l2);
                    ab += ob * k;
                    g1[0] += ob * k * dx;
                    g1[1] += ob * k * dy;
                    g1[2] += ob * k * dz;
                }
                s.z[j] = ab;
                for (int a = 0; a < 3; ++a) g1[a] *= s.alpha[j] / l2;
                const int64_t gi = c.bw.gidx[base + j];
                for (int a = 0; a < 3; ++a) atomicAdd(&c.bw.dL_dX[3 * gi + a], g1[a]);
            }
            __syncthreads();
            chol_solve(s, s.A, Nt, s.w);  // lambda = A^-1 abar -> s.w
            for (int j = tid; j < N; j += nt) {
                double g2[3] = {0.0, 0.0, 0.0};
                const double lj = s.w[j], aj = s.alpha[j];
                for (int i = 0; i < N; ++i) {
                    if (i == j) continue;
                    double dx = s.X[3 * i] - s.X[3 * j], dy = s.X[3 * i + 1] - s.X[3 * j + 1],
                           dz = s.X[3 * i + 2] - s.X[3 * j + 2];
                    double k = exp(-(dx * dx + dy * dy + dz * dz) * c.P.inv2l2);
                    double cf = (s.w[i] * aj + lj * s.alpha[i]) * k;
                    g2[0] -= cf * dx;
                    g2[1] -= cf * dy;
                    g2[2] -= cf * dz;
                }
                const int64_t gi = c.bw.gidx[base + j];
                for (int a = 0; a < 3; ++a) atomicAdd(&c.bw.dL_dX[3 * gi + a], g2[a] / l2);
            }
        }
        __syncthreads();
    }
}

__global__ void k_hist_n(const int64_t* inst_off, int64_t n, int* hist) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int N = (int)(inst_off[i + 1] - inst_off[i]);
    atomicAdd(&hist[min(N, 1024)], 1);
}

// Queries of each size bucket (N > 224, > 128, > 64, > 32, the rest), for the chunk planning.
__global__ void k_bucket_queries(const int64_t* inst_off, const int64_t* q_off, int64_t n, unsigned long long* qsum) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t N = inst_off[i + 1] - inst_off[i];
    const int bk = N > 224 ? 0 : N > 128 ? 1 : N > 64 ? 2 : N > 32 ? 3 : 4;
    atomicAdd(&qsum[bk], (unsigned long long)(q_off[i + 1] - q_off[i]));
}

// order[] sorted by increasing N via the prefix of the histogram
__global__ void k_order_n(const int64_t* inst_off, int64_t n, int* cursor, int32_t* order) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int N = (int)(inst_off[i + 1] - inst_off[i]);
    int pos = atomicAdd(&cursor[min(N, 1024)], 1);
    order[pos] = (int32_t)i;
}

__global__ void k_or_err(int* err, int bits) { atomicOr(err, bits); }

// Device bucket plan (graph mode): cursor[N] = first position of size N in decreasing-N
// order; plan[b] = instances of bucket b, plan[5 + b] = its first position.
__global__ void k_plan_buckets(const int* hist, int* cursor, int* plan) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int N = 1024; N >= 0; --N) {
        cursor[N] = run;
        run += hist[N];
    }
    const int lo[5] = {225, 129, 65, 33, 0}, hi[5] = {1024, 224, 128, 64, 32};
    int off = 0;
    for (int b = 0; b < 5; ++b) {
        int cnt = 0;
        for (int N = lo[b]; N <= hi[b]; ++N) cnt += hist[N];
        plan[b] = cnt;
        plan[5 + b] = off;
        off += cnt;
    }
}

// Work items of the solve launches: where the evaluation is heavy (variance, surface
// properties), a bucket with few instances is split into chunks of qc queries (chunk_size) so
// that its queries spread over the GPU; each chunk fits its instance again.  cap[b] > 0
// bounds qc (the rows a bordered factorisation appends).  chunk_q[b] receives qc (0: no
// split; taken from a.qc when the host decided); chunk_off[k]
// the number of work items of the order before instance k, chunk_off[n] the total.  The
// buckets are contiguous in the order: from the device plan in graph mode, else from a.
struct ChunkPlanArgs {
    int off[5], cnt[5], slots[5], cap[5];
    int heavy;
    int decided, qc[5];  // decided: the chunk sizes qc were chosen on the host (same rule)
};
constexpr int kMinChunk = 64, kMinChunksPer = 8;
// Queries per work item of a bucket of cnt instances with tq queries in all, launched on slots
// CTAs; cap > 0 bounds it; 0: no bound (one work item per instance).  A bucket that holds at
// most half as many instances as CTAs is split into chunks of ceil(tq / slots) queries, at
// least kMinChunk, when that gives its instances kMinChunksPer chunks on average: for fewer,
// fitting each chunk again costs more than the spread gains.
__host__ __device__ inline int chunk_size(bool heavy, int cnt, int slots, int cap, long long tq) {
    int qc = cap;
    if (heavy && cnt > 0 && 2 * (long long)cnt <= slots) {
        long long want = (tq + slots - 1) / slots;
        if (want < kMinChunk) want = kMinChunk;
        if (tq >= (long long)kMinChunksPer * want * cnt) {
            if (qc > 0 && qc < want) want = qc;
            qc = (int)(want < INT32_MAX ? want : INT32_MAX);
        }
    }
    return qc;
}
__global__ void k_chunk_plan(const int32_t* order, int n, const int64_t* inst_off, const int64_t* q_off,
                             const int* plan, ChunkPlanArgs a, int* chunk_q, int* chunk_off) {
    __shared__ long long wq[32];
    __shared__ int wsum[32];
    __shared__ int carry, s_qc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    if (tid == 0) carry = 0;
    for (int bk = 0; bk < 5; ++bk) {
        const int off = plan ? plan[5 + bk] : a.off[bk], cnt = plan ? plan[bk] : a.cnt[bk];
        // the bucket's queries
        long long q = 0;
        for (int k = tid; k < cnt; k += blockDim.x) {
            const int I = order[off + k];
            q += q_off[I + 1] - q_off[I];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (lane == 0) wq[warp] = q;
        __syncthreads();
        if (tid == 0) {
            long long tq = 0;
            for (int w = 0; w < nwarp; ++w) tq += wq[w];
            int qc = a.decided ? a.qc[bk] : chunk_size(a.heavy != 0, cnt, a.slots[bk], a.cap[bk], tq);
            chunk_q[bk] = qc;
            s_qc = qc;
        }
        __syncthreads();
        const int qc = s_qc;
        // exclusive scan of the chunk counts, continuing the running total
        for (int b0 = 0; b0 < cnt; b0 += blockDim.x) {
            const int k = b0 + tid;
            int v = 0;
            if (k < cnt) {
                const int I = order[off + k];
                const int64_t nq = q_off[I + 1] - q_off[I];
                v = qc > 0 ? (int)max((int64_t)1, (nq + qc - 1) / qc) : 1;
            }
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[warp] = x;
            __syncthreads();
            if (warp == 0) {
                int t = lane < nwarp ? wsum[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t += y;
                }
                wsum[lane] = t;
            }
            __syncthreads();
            const int excl = carry + (warp > 0 ? wsum[warp - 1] : 0) + x - v;
            if (k < cnt) chunk_off[off + k] = excl;
            __syncthreads();
            if (tid == blockDim.x - 1) carry = excl + v;
            __syncthreads();
        }
    }
    if (tid == 0) chunk_off[n] = carry;
}

__global__ void k_reverse_i32(const int32_t* in, int32_t* out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[n - 1 - i];
}

// A workspace allocation failed: record it in the error word and launch nothing else.
int alloc_failed(int* err_dev, cudaStream_t st) {
    cudaGetLastError();
    k_or_err<<<1, 1, 0, st>>>(err_dev, kErrAlloc);
    note_launch();
    return -2;
}

}  // namespace

// One persistent launch of k_solve over instances in the given order with caller-provided
// scratch (no allocation): A in shared memory (npad <= 224), variance columns in ws_v
// (max_grid * npad * threads doubles), work counter *counter zeroed by the caller.
int solve_launch_static(const SolveBatch& b, const DevParams& P, int* err_dev, int npad, int threads, int max_grid,
                        int* counter, const int32_t* order, double* ws_v, cudaStream_t st) {
    SolveCtx c;
    c.plan = nullptr;
    c.bucket = 0;
    c.ws_e = nullptr;
    c.ws_e_stride = 0;
    c.b = b;
    c.P = P;
    c.err = err_dev;
    c.counter = counter;
    c.order = order;
    c.inst_base = 0;
    c.n_work = (int)b.n_inst;
    c.npad = npad;
    c.a_in_smem = 1;
    c.stage_panel = 1;
    c.ws_a = nullptr;
    c.ws_a_stride = 0;
    const size_t shm = smem_bytes(npad, 1, 0, 1, b.Xi != nullptr);
    if (cudaFuncSetAttribute(k_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm) != cudaSuccess)
        return -1;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<false>, threads, shm);
    const int grid = (int)std::min<int64_t>(std::min<int64_t>(b.n_inst, (int64_t)n_sm * std::max(per_sm, 1)), max_grid);
    c.ws_v_stride = (int64_t)npad * threads;
    c.ws_v = ws_v;
    k_solve<false><<<grid, threads, shm, st>>>(c);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

namespace {

using SolveKernel = void (*)(SolveCtx);

SolveKernel pick_solve(bool props, bool emu) {
    if (props) return emu ? k_solve_emu<true> : k_solve<true>;
    return emu ? k_solve_emu<false> : k_solve<false>;
}

// seven bf16 slices of a block's columns, the row scale, and one row of diagonal-tile inverses
constexpr int64_t kEmuBytesPerRow = 7 * 8 * kEB * 2 + 8 + 64;

// Chunk planning of a solve (see k_chunk_plan): heavy evaluation, and the bordered emulated
// bucket's bound (kBorderQ queries appended at a time).  False when no launch splits.
bool chunk_args(const SolveBatch& b, const DevParams& P, bool bw, ChunkPlanArgs& a) {
    a = ChunkPlanArgs{};
    a.heavy = !bw && (b.want_var || b.nprop > 0);
    a.cap[0] = (!bw && P.emulate && b.want_var) ? kBorderQ : 0;
    a.cap[1] = a.cap[2] = a.cap[3] = a.cap[0];  // the emulated buckets
    return a.heavy != 0;
}

// Emulated launch with the latent variance: the queries of an instance (up to kBorderQ) are
// appended to its matrix, which is padded to a multiple of 32 rows (see fit_instance); the
// workspaces hold npad + kBorderQ rows.  Otherwise npad rows.
void emu_rows_for(bool emu, const SolveBatch& b, int& npad, int& qmax, int& nrow) {
    qmax = 0;
    if (emu && b.want_var) {
        npad = (npad + 31) & ~31;
        qmax = kBorderQ;
    }
    nrow = npad + qmax;
}

// The emulated kernel's shared memory (about 100 KB at N = 1024) fits twice per SM only in the
// largest shared-memory configuration; ask for it (a preference, so a failure is harmless).
void set_emu_carveout(SolveKernel k) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        cudaGetLastError();
}

// Resident CTAs per SM of the emulated kernel.  The occupancy calculator reports one CTA per SM
// for any kernel that allocates tensor memory, while the SM runs as many as their registers,
// shared memory and tensor memory allow (each CTA holds kEmuTmemCols of the 512 columns), so
// the bound is computed from those resources.
int emu_ctas_per_sm(SolveKernel k, int threads, size_t shm) {
    cudaFuncAttributes fa{};
    int dev = 0, regs_sm = 65536, smem_sm = 0, thr_sm = 2048;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int warps = (threads + 31) / 32;
    const int regs_cta = warps * ((fa.numRegs * 32 + 255) & ~255);  // allocated per warp in units of 256
    const size_t smem_cta = shm + fa.sharedSizeBytes + 1024;        // 1 KB reserved per CTA
    int n = kEmuCtasPerSm;
    n = std::min(n, regs_cta > 0 ? regs_sm / regs_cta : n);
    n = std::min(n, (int)(smem_sm / std::max<size_t>(smem_cta, 1)));
    n = std::min(n, thr_sm / std::max(threads, 1));
    return std::max(n, 1);
}

}  // namespace

void graph_cache_destroy(GraphCache& gc) {
    for (auto& e : gc.exec)
        if (e) cudaGraphExecDestroy(e);
    if (gc.e0) cudaEventDestroy(gc.e0);
    if (gc.e1) cudaEventDestroy(gc.e1);
    if (gc.t0) cudaEventDestroy(gc.t0);
    if (gc.t1) cudaEventDestroy(gc.t1);
    if (gc.gs) cudaStreamDestroy(gc.gs);
    gc = GraphCache{};
}

namespace {

void add_stats(SolveStats* stats, const std::vector<int>& h) {
    if (!stats) return;
    for (int N = 0; N <= 1024; ++N) {
        int bk = N <= 32 ? 0 : N <= 64 ? 1 : N <= 128 ? 2 : N <= 256 ? 3 : 4;
        stats->bucket_count[bk] += h[N];
        stats->sum_n3 += (double)h[N] * N * N * N;
        stats->sum_n2 += (double)h[N] * N * N;
    }
}

// Graph mode: the whole solve -- size histogram, bucket plan, decreasing-size order and one
// persistent launch per size bucket -- is planned on the device, captured as a CUDA graph on
// the map's private stream and replayed through a cached executable graph (updated in place
// when only the arguments changed).  Launch shapes come from the map's configuration, sized
// for the largest N the batch can hold; CTAs of a bucket with no work exit at once.  Returns
// 0, -1 when a CUDA call failed, or -2 when a workspace could not be allocated (nothing was
// launched; kErrAlloc is set in *err_dev).
int solve_batch_graph(const SolveBatch& b, const DevParams& P, int* err_dev, cudaStream_t st, Arena& ar,
                      SolveStats* stats, bool profile, const SolveConfig* cfg, GraphCache* gc) {
    const int64_t n = b.n_inst;
    if (!gc->gs) {
        if (cudaStreamCreateWithFlags(&gc->gs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&gc->e0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&gc->e1, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&gc->t0) != cudaSuccess || cudaEventCreate(&gc->t1) != cudaSuccess)
            return -1;
    }
    const bool props = b.nprop > 0;
    const int T = 256;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int maxn = std::min(std::max(b.max_n, 1), 1024);
    const int lo[5] = {225, 129, 65, 33, 0}, hi[5] = {1024, 224, 128, 64, 32};
    struct Shape {
        int npad, smem_a, stage, threads, grid, qmax, nrow;
        size_t shm;
        bool live, emu;
        SolveKernel kern;
    } sh[5];
    for (int i = 0; i < 5; ++i) {
        Shape& s = sh[i];
        s.live = maxn >= lo[i];
        s.npad = std::max((std::min(hi[i], maxn) + 7) & ~7, 8);
        s.smem_a = i > (P.emulate ? 3 : 0);  // emulated: the buckets above 32 points
        s.emu = !s.smem_a && P.emulate;
        emu_rows_for(s.emu, b, s.npad, s.qmax, s.nrow);
        s.stage = s.smem_a ? 1 : (s.emu ? 0 : cfg->stage_panel);
        s.threads = s.emu ? kEmuThreads : cfg->threads[i];
        s.shm = smem_bytes(s.npad, s.smem_a, b.nprop, s.stage, b.Xi != nullptr, false, s.emu);
        s.kern = pick_solve(props, s.emu);
    }
    // buckets share a kernel: its shared-memory limit is the largest of the live buckets that
    // launch it, set before any occupancy query or captured launch
    for (int i = 0; i < 5; ++i) {
        if (!sh[i].live) continue;
        if (sh[i].emu) set_emu_carveout(sh[i].kern);
        size_t shm_max = 0;
        for (int j = 0; j < 5; ++j)
            if (sh[j].live && sh[j].kern == sh[i].kern) shm_max = std::max(shm_max, sh[j].shm);
        if (cudaFuncSetAttribute(sh[i].kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_max) != cudaSuccess)
            return -1;
    }
    ChunkPlanArgs ca;
    const bool chunks = chunk_args(b, P, false, ca);
    int64_t ws_a_need = 0, ws_v_need = 0, ws_e_need = 0;
    for (int i = 0; i < 5; ++i) {
        Shape& s = sh[i];
        if (!s.live) continue;
        int per_sm = 0;
        if (s.emu) {
            per_sm = emu_ctas_per_sm(s.kern, s.threads, s.shm);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, s.kern, s.threads, s.shm);
            per_sm = std::max(per_sm, 1);
            if (cfg->per_sm[i] > 0) per_sm = std::min(per_sm, cfg->per_sm[i]);
        }
        s.grid = (int)std::min<int64_t>(n, (int64_t)n_sm * per_sm);
        ca.slots[i] = s.grid;
        if (!s.smem_a) ws_a_need = std::max<int64_t>(ws_a_need, n_tiles(s.nrow / 8) * 64 * s.grid);
        if (b.want_var) ws_v_need = std::max<int64_t>(ws_v_need, (int64_t)s.npad * s.threads * s.grid);
        if (s.emu) ws_e_need = std::max<int64_t>(ws_e_need, (int64_t)s.nrow * kEmuBytesPerRow * s.grid);
    }
    // every buffer exists before the capture starts (allocation is not captured)
    int* hist = (int*)ar.get(Arena::kHist, sizeof(int) * 2 * 1025, st);
    int32_t* order = (int32_t*)ar.get(Arena::kOrder, sizeof(int32_t) * n, st);
    int* counters = (int*)ar.get(Arena::kCounters, sizeof(int) * 16, st);
    double* ws_a = ws_a_need ? (double*)ar.get(Arena::kWs0, sizeof(double) * ws_a_need, st) : nullptr;
    double* ws_v = ws_v_need ? (double*)ar.get(Arena::kWs1, sizeof(double) * ws_v_need, st) : nullptr;
    uint8_t* ws_e = ws_e_need ? (uint8_t*)ar.get(Arena::kWs3, ws_e_need, st) : nullptr;
    int* chunk_off = chunks ? (int*)ar.get(Arena::kChunks, sizeof(int) * (n + 1 + 5), st) : nullptr;
    if (!hist || !order || !counters || (ws_a_need && !ws_a) || (ws_v_need && !ws_v) || (ws_e_need && !ws_e) ||
        (chunks && !chunk_off))
        return alloc_failed(err_dev, st);
    int* chunk_q = chunk_off ? chunk_off + n + 1 : nullptr;
    int* cursor = hist + 1025;
    int* plan = counters + 5;
    cudaStream_t gs = gc->gs;
    if (cudaEventRecord(gc->e0, st) != cudaSuccess || cudaStreamWaitEvent(gs, gc->e0, 0) != cudaSuccess) return -1;
    if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
    fill_i32(hist, 0, 1025, gs);
    fill_i32(counters, 0, 5, gs);
    k_hist_n<<<(unsigned)((n + T - 1) / T), T, 0, gs>>>(b.inst_off, n, hist);
    note_launch();
    k_plan_buckets<<<1, 32, 0, gs>>>(hist, cursor, plan);
    note_launch();
    k_order_n<<<(unsigned)((n + T - 1) / T), T, 0, gs>>>(b.inst_off, n, cursor, order);
    note_launch();
    if (chunk_off) {
        k_chunk_plan<<<1, 1024, 0, gs>>>(order, (int)n, b.inst_off, b.q_off, plan, ca, chunk_q, chunk_off);
        note_launch();
    }
    for (int i = 0; i < 5; ++i) {
        const Shape& s = sh[i];
        if (!s.live) continue;
        SolveCtx c;
        c.chunk_off = chunk_off;
        c.chunk_q = chunk_q ? chunk_q + i : nullptr;
        c.b = b;
        c.P = P;
        c.err = err_dev;
        c.counter = counters + i;
        c.order = order;
        c.inst_base = 0;
        c.n_work = 0;
        c.plan = plan;
        c.bucket = i;
        c.npad = s.npad;
        c.a_in_smem = s.smem_a;
        c.stage_panel = s.stage;
        c.qmax = s.qmax;
        c.nrow = s.nrow;
        c.ws_a_stride = s.smem_a ? 0 : n_tiles(s.nrow / 8) * 64;
        c.ws_a = s.smem_a ? nullptr : ws_a;
        c.ws_v_stride = (int64_t)s.npad * s.threads;
        c.ws_v = ws_v;
        c.ws_e_stride = s.emu ? (int64_t)s.nrow * kEmuBytesPerRow : 0;
        c.ws_e = s.emu ? ws_e : nullptr;
        s.kern<<<s.grid, s.threads, s.shm, gs>>>(c);
        note_launch();
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamEndCapture(gs, &graph) != cudaSuccess || !graph) return -1;
    cudaGraphExec_t& ex = gc->exec[props ? 1 : 0];
    if (ex) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ex, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    }
    if (!ex) {
        if (cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) {
            ex = nullptr;
            cudaGraphDestroy(graph);
            return -1;
        }
        ++gc->instantiations;
    }
    cudaGraphDestroy(graph);
    if (profile) cudaEventRecord(gc->t0, gs);
    if (cudaGraphLaunch(ex, gs) != cudaSuccess) return -1;
    ++gc->replays;
    if (profile) cudaEventRecord(gc->t1, gs);
    if (cudaEventRecord(gc->e1, gs) != cudaSuccess || cudaStreamWaitEvent(st, gc->e1, 0) != cudaSuccess) return -1;
    // statistics: the size histogram, read once after the solve
    std::vector<int> h(1025);
    cudaMemcpyAsync(h.data(), hist, sizeof(int) * 1025, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    add_stats(stats, h);
    if (profile && stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, gc->t0, gc->t1);
        stats->t_solve_ms += ms;
    }
    return 0;
}

}  // namespace

int solve_batch(const SolveBatch& b, const DevParams& P, int* err_dev, cudaStream_t st, Arena& ar, SolveStats* stats,
                 const BackwardBatch* bw, bool profile, int launch, const SolveConfig* cfg, GraphCache* gc) {
    const SolveConfig dflt;
    if (!cfg) cfg = &dflt;
    const int64_t n = b.n_inst;
    if (n <= 0) return 0;
    if (launch == VGP_LAUNCH_GRAPH && !bw && gc) {
        const int rc = solve_batch_graph(b, P, err_dev, st, ar, stats, profile, cfg, gc);
        if (rc == -2) return rc;
        if (rc != 0) {
            // leave the capture stream usable and the error visible to the caller
            cudaGraph_t g = nullptr;
            cudaStreamCaptureStatus cs;
            if (gc->gs && cudaStreamIsCapturing(gc->gs, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
                cudaStreamEndCapture(gc->gs, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            k_or_err<<<1, 1, 0, st>>>(err_dev, kErrLaunch);
            note_launch();
            return -1;
        }
        return 0;
    }
    // size histogram (and, for chunk planning, each bucket's queries) and decreasing-size order
    ChunkPlanArgs ca;
    const bool heavy = chunk_args(b, P, bw != nullptr, ca);
    int* hist = (int*)ar.get(Arena::kHist, sizeof(int) * 2 * 1025 + sizeof(unsigned long long) * 5, st);
    if (!hist) return alloc_failed(err_dev, st);
    int* cursor = hist + 1025;
    unsigned long long* qsum = reinterpret_cast<unsigned long long*>(hist + 2 * 1025);
    cudaMemsetAsync(hist, 0, sizeof(int) * 1025, st);
    const int T = 256;
    k_hist_n<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(b.inst_off, n, hist);
    note_launch();
    unsigned long long hq[5] = {0, 0, 0, 0, 0};
    if (heavy) {
        cudaMemsetAsync(qsum, 0, sizeof(hq), st);
        k_bucket_queries<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(b.inst_off, b.q_off, n, qsum);
        note_launch();
    }
    std::vector<int> h(1025);
    cudaMemcpyAsync(h.data(), hist, sizeof(int) * 1025, cudaMemcpyDeviceToHost, st);
    if (heavy) cudaMemcpyAsync(hq, qsum, sizeof(hq), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    std::vector<int> start(1026, 0);
    for (int i = 0; i < 1025; ++i) start[i + 1] = start[i] + h[i];
    cudaMemcpyAsync(cursor, start.data(), sizeof(int) * 1025, cudaMemcpyHostToDevice, st);
    int32_t* order_inc = (int32_t*)ar.get(Arena::kOrder, sizeof(int32_t) * 2 * n, st);
    if (!order_inc) return alloc_failed(err_dev, st);
    int32_t* order = order_inc + n;
    k_order_n<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(b.inst_off, n, cursor, order_inc);
    note_launch();
    k_reverse_i32<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(order_inc, order, (int)n);
    note_launch();
    add_stats(stats, h);
    int* chunk_off = nullptr;
    int* chunk_q = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (profile) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, st);
    }
    // size buckets, largest first: A in global workspace above 224, in shared memory below
    struct Bucket {
        int lo, hi, smem_a, threads;
    };
    // with the emulated updates every bucket above 32 points runs the emulated kernel (A in
    // global memory): a single 32-column block leaves it nothing to gain below
    const int emu_mid = P.emulate && !bw ? 0 : 1;
    const Bucket buckets[] = {{225, 1024, 0, cfg->threads[0]}, {129, 224, emu_mid, cfg->threads[1]},
                              {65, 128, emu_mid, cfg->threads[2]}, {33, 64, emu_mid, cfg->threads[3]},
                              {0, 32, 1, cfg->threads[4]}};
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (launch == VGP_LAUNCH_PER_INSTANCE && !bw) {
        // the plain comparison form: one launch per instance, in instance order, one CTA each
        // workspaces sized for the largest instance (N <= 1024, at most 512 threads, appended
        // query rows of the emulated kernel)
        constexpr int kRowsMax = 1024 + kBorderQ;
        int* ctr = (int*)ar.get(Arena::kCounters, sizeof(int) * n, st);
        uint8_t* ws_e = P.emulate ? (uint8_t*)ar.get(Arena::kWs3, kRowsMax * kEmuBytesPerRow, st) : nullptr;
        double* ws_a = (double*)ar.get(Arena::kWs0, sizeof(double) * n_tiles(kRowsMax / 8) * 64, st);
        double* ws_v = b.want_var ? (double*)ar.get(Arena::kWs1, sizeof(double) * 1024 * 512, st) : nullptr;
        if (!ctr || !ws_a || (P.emulate && !ws_e) || (b.want_var && !ws_v)) {
            if (profile) {
                cudaEventDestroy(ev0);
                cudaEventDestroy(ev1);
            }
            return alloc_failed(err_dev, st);
        }
        cudaMemsetAsync(ctr, 0, sizeof(int) * n, st);
        std::vector<int64_t> off(n + 1);
        cudaMemcpyAsync(off.data(), b.inst_off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        for (int64_t I = 0; I < n; ++I) {
            const int N = (int)(off[I + 1] - off[I]);
            SolveCtx c;
            c.plan = nullptr;
            c.bucket = 0;
            c.ws_e = nullptr;
            c.ws_e_stride = 0;
            c.b = b;
            c.P = P;
            c.err = err_dev;
            c.counter = ctr + I;
            c.order = nullptr;
            c.inst_base = (int)I;
            c.n_work = 1;
            c.npad = std::max((N + 7) & ~7, 8);
            c.a_in_smem = c.npad <= 224;
            const bool emu = !c.a_in_smem && P.emulate;
            emu_rows_for(emu, b, c.npad, c.qmax, c.nrow);
            c.stage_panel = emu ? 0 : 1;
            const int threads = emu ? kEmuThreads : c.npad <= 32 ? 64 : c.npad <= 64 ? 128 : c.npad <= 128 ? 256 : 512;
            const size_t shm = smem_bytes(c.npad, c.a_in_smem, b.nprop, c.stage_panel, b.Xi != nullptr, false, emu);
            auto ks = pick_solve(b.nprop > 0, emu);
            c.ws_e_stride = emu ? (int64_t)c.nrow * kEmuBytesPerRow : 0;
            c.ws_e = emu ? ws_e : nullptr;
            cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            c.ws_a_stride = c.a_in_smem ? 0 : n_tiles(c.nrow / 8) * 64;
            c.ws_a = c.a_in_smem ? nullptr : ws_a;
            c.ws_v_stride = (int64_t)c.npad * threads;
            c.ws_v = ws_v;
            ks<<<1, threads, shm, st>>>(c);
            note_launch();
        }
        if (profile) {
            cudaEventRecord(ev1, st);
            cudaEventSynchronize(ev1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev0, ev1);
            if (stats) stats->t_solve_ms += ms;
            cudaEventDestroy(ev0);
            cudaEventDestroy(ev1);
        }
        return 0;
    }
    // a bucket's launch: shapes, kernel and resident CTAs per SM
    struct Launch {
        int npad, qmax, nrow, threads, stage, per_sm;
        size_t shm;
        bool emu;
        SolveKernel kern;
    };
    auto bucket_nmax = [&](int i, int& cnt) {
        int nmax = 0;
        cnt = 0;
        for (int N = buckets[i].lo; N <= buckets[i].hi; ++N) {
            cnt += h[N];
            if (h[N]) nmax = N;
        }
        return nmax;
    };
    auto bucket_launch = [&](int i, int nmax) {
        const Bucket& bk = buckets[i];
        Launch L;
        L.npad = std::max((nmax + 7) & ~7, 8);
        L.emu = !bw && !bk.smem_a && P.emulate;
        emu_rows_for(L.emu, b, L.npad, L.qmax, L.nrow);
        L.threads = L.emu ? kEmuThreads : bk.threads;
        L.stage = bk.smem_a ? 1 : (L.emu ? 0 : cfg->stage_panel);
        L.shm = smem_bytes(L.npad, bk.smem_a, bw ? 0 : b.nprop, L.stage, b.Xi != nullptr, bw != nullptr, L.emu);
        L.kern = bw ? k_backward : pick_solve(b.nprop > 0, L.emu);
        cudaFuncSetAttribute(L.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.shm);
        if (L.emu) set_emu_carveout(L.kern);
        L.per_sm = 0;
        if (L.emu) {
            L.per_sm = emu_ctas_per_sm(L.kern, L.threads, L.shm);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L.per_sm, L.kern, L.threads, L.shm);
            L.per_sm = std::max(L.per_sm, 1);
            if (cfg->per_sm[i] > 0) L.per_sm = std::min(L.per_sm, cfg->per_sm[i]);
        }
        return L;
    };
    int* counters = (int*)ar.get(Arena::kCounters, sizeof(int) * 8, st);
    bool chunks = false;
    if (heavy) {
        // the buckets' ranges of the order, their resident CTAs (as the launches below) and
        // chunk sizes; work items are planned only where some bucket has more than its instances
        int off = 0;
        for (int i = 0; i < 5; ++i) {
            int cnt = 0;
            const int nmax = bucket_nmax(i, cnt);
            ca.off[i] = off;
            ca.cnt[i] = cnt;
            off += cnt;
            ca.slots[i] = cnt > 0 ? n_sm * bucket_launch(i, nmax).per_sm : 0;
            ca.qc[i] = chunk_size(true, cnt, ca.slots[i], ca.cap[i], (long long)hq[i]);
            chunks = chunks || (cnt > 0 && ca.qc[i] > 0);
        }
        ca.decided = 1;
    }
    if (chunks) {
        chunk_off = (int*)ar.get(Arena::kChunks, sizeof(int) * (n + 1 + 5), st);
        if (chunk_off) {
            chunk_q = chunk_off + n + 1;
            k_chunk_plan<<<1, 1024, 0, st>>>(order, (int)n, b.inst_off, b.q_off, nullptr, ca, chunk_q, chunk_off);
            note_launch();
        }
    }
    if (!counters || (chunks && !chunk_off)) {
        if (profile) {
            cudaEventDestroy(ev0);
            cudaEventDestroy(ev1);
        }
        return alloc_failed(err_dev, st);
    }
    cudaMemsetAsync(counters, 0, sizeof(int) * 8, st);
    int done = 0;  // instances already assigned (from the large end)
    int bi = 0;
    for (const Bucket& bk : buckets) {
        int cnt = 0;
        const int nmax = bucket_nmax(bi, cnt);
        if (cnt == 0) {
            ++bi;
            continue;
        }
        SolveCtx c;
        c.plan = nullptr;
        c.bucket = 0;
        c.ws_e = nullptr;
        c.ws_e_stride = 0;
        c.b = b;
        c.P = P;
        c.err = err_dev;
        c.counter = counters + bi;
        c.order = order + done;
        c.inst_base = 0;
        c.n_work = cnt;
        c.chunk_off = chunk_off ? chunk_off + done : nullptr;
        c.chunk_q = chunk_q ? chunk_q + bi : nullptr;
        const Launch L = bucket_launch(bi, nmax);
        c.npad = L.npad;
        c.qmax = L.qmax;
        c.nrow = L.nrow;
        c.a_in_smem = bk.smem_a;
        const bool emu = L.emu;
        const int threads = L.threads;
        c.stage_panel = L.stage;
        if (bw) c.bw = *bw;
        const size_t shm = L.shm;
        auto kern = L.kern;
        const int per_sm = L.per_sm;
        // a split bucket keeps every resident CTA busy; otherwise one CTA per instance at most
        const bool split = chunk_off && ca.qc[bi] > 0;
        const int grid = (int)std::min<int64_t>(split ? INT32_MAX : cnt, (int64_t)n_sm * per_sm);
        c.ws_a_stride = c.a_in_smem ? 0 : n_tiles(c.nrow / 8) * 64;
        c.ws_a = c.a_in_smem ? nullptr : (double*)ar.get(Arena::kWs0, sizeof(double) * c.ws_a_stride * grid, st);
        c.ws_v_stride = (int64_t)c.npad * threads;
        c.ws_v = (b.want_var && !bw) ? (double*)ar.get(Arena::kWs1, sizeof(double) * c.ws_v_stride * grid, st) : nullptr;
        c.ws_e_stride = emu ? (int64_t)c.nrow * kEmuBytesPerRow : 0;
        c.ws_e = emu ? (uint8_t*)ar.get(Arena::kWs3, c.ws_e_stride * grid, st) : nullptr;
        if ((!c.a_in_smem && !c.ws_a) || (b.want_var && !bw && !c.ws_v) || (emu && !c.ws_e)) {
            if (profile) {
                cudaEventDestroy(ev0);
                cudaEventDestroy(ev1);
            }
            return alloc_failed(err_dev, st);
        }
        cudaEvent_t b0 = nullptr, b1 = nullptr;
        if (profile) {
            cudaEventCreate(&b0);
            cudaEventCreate(&b1);
            cudaEventRecord(b0, st);
        }
        kern<<<grid, threads, shm, st>>>(c);
        note_launch();
        if (profile) {
            cudaEventRecord(b1, st);
            cudaEventSynchronize(b1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, b0, b1);
            if (stats) stats->t_bucket_ms[bi] += ms;
            cudaEventDestroy(b0);
            cudaEventDestroy(b1);
        }
        done += cnt;
        ++bi;
    }
    if (profile) {
        cudaEventRecord(ev1, st);
        cudaEventSynchronize(ev1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (stats) stats->t_solve_ms += ms;
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    return 0;
}

namespace {
// One pair of FP32 world coordinates per thread: the emulated kernel's mixed-precision kernel
// value in the fixed point.
__global__ void k_kfix_probe(const float* xa, const float* xb, long long* out, int64_t n, DevParams P) {
    __shared__ float2 tab[256];
    for (int j = threadIdx.x; j < 256; j += blockDim.x) {
        float h, l;
        split_pair(P.exp_tab[j], h, l);
        tab[j] = make_float2(h, l);
    }
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a[3] = {xa[3 * i], xa[3 * i + 1], xa[3 * i + 2]};
    const float b[3] = {xb[3 * i], xb[3 * i + 1], xb[3 * i + 2]};
    out[i] = kfix_ff(a, b, P.inv2l2_hi, P.inv2l2_lo, tab);
}
}  // namespace

int debug_kernel_fix(const DevParams& P, const float* xa, const float* xb, int64_t n, long long* out,
                     cudaStream_t st) {
    if (n <= 0) return 0;
    k_kfix_probe<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xa, xb, out, n, P);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace vgp
