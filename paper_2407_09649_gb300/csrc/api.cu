// api.cu -- the C ABI (include/vgpdf.h): map and frame handles, device memory, and the
// orchestration of the L-GPDF frame (Sec. IV-A/B), fusion (Sec. IV-C) and G-GPDF queries
// (Sec. IV-D) over the kernels of grid.cu and solve.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "grid.h"
#include "mesh.h"

using namespace vgp;

// --------------------------------------------------------------------------------------
// errors
// --------------------------------------------------------------------------------------
static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

namespace vgp {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace vgp

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) return fail(VGP_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// --------------------------------------------------------------------------------------
// arena
// --------------------------------------------------------------------------------------
namespace vgp {
void* Arena::get(Slot s, size_t bytes, cudaStream_t st) {
    bytes = std::max<size_t>(bytes, 256);
    if (size_[s] >= bytes) return ptr_[s];
    if (ptr_[s]) cudaFreeAsync(ptr_[s], st);
    size_t want = std::max(bytes, size_[s] + size_[s] / 2);
    void* p = nullptr;
    if (cudaMallocAsync(&p, want, st) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            ptr_[s] = nullptr;
            size_[s] = 0;
            return nullptr;
        }
        want = bytes;
    }
    ptr_[s] = p;
    size_[s] = want;
    return p;
}
void Arena::release_all(cudaStream_t st) {
    for (int i = 0; i < kNumSlots; ++i) {
        if (ptr_[i]) cudaFreeAsync(ptr_[i], st);
        ptr_[i] = nullptr;
        size_[i] = 0;
    }
}
Arena::~Arena() {
    for (int i = 0; i < kNumSlots; ++i)
        if (ptr_[i]) cudaFree(ptr_[i]);
}
}  // namespace vgp

static uint32_t pow2_at_least(int64_t n) {
    uint64_t c = 64;
    while ((int64_t)c < n) c <<= 1;
    if (c > (1ull << 31)) c = 1ull << 31;
    return (uint32_t)c;
}

// --------------------------------------------------------------------------------------
// handles
// --------------------------------------------------------------------------------------
struct vgp_map {
    vgp_params prm{};
    DevParams P{};
    int device = 0;
    Arena ar;
    int* dev_words = nullptr;  // [0] err, [1] n_valid, [2] count, [3] pool_count, [4] orphan
    double* tables = nullptr;  // exp_neg table (256) + lattice kernel table (kLatticeTable), FP64
    float* tables_f = nullptr; // lattice kernel table in FP32
    int* host_words = nullptr; // pinned mirror
    // global grid
    Table g;
    int32_t* g_slot2pool = nullptr;
    int pool_cap = 0;
    unsigned long long* g_known = nullptr;
    double* g_D = nullptr;
    double* g_V = nullptr;
    int32_t* g_flags = nullptr;
    double* g_C = nullptr;  // fused surface properties [pool][512][n_props] (Eq. 6, Sec. IV-C)
    double* g_W = nullptr;  // their variances / weights [pool][512]; NaN: none fused
    int g_leaves = 0;
    // surface
    float* s_pts = nullptr;
    int64_t s_n = 0, s_pts_cap = 0;
    Table s_tab;
    int32_t* s_slot2leaf = nullptr;
    int s_nl = 0;
    int64_t* s_off = nullptr;
    int32_t* s_idx = nullptr;
    int64_t s_idx_cap = 0, s_off_cap = 0;
    bool has_surface = false;
    // G-GPDF training set kept per leaf from the grid's zero crossings (vgp_update_surface)
    float* ps_pts = nullptr;
    float* ps_tmp = nullptr;
    int64_t ps_n = 0, ps_cap = 0, ps_tmp_cap = 0;
    uint8_t* mc_tab = nullptr;  // marching-cubes table: 256 x 16 cell edges, then 256 counts
    vgp_stats stats{};
    SolveConfig cfg;  // launch shape per size bucket (vgp_autotune)
    GraphCache gcache;  // VGP_LAUNCH_GRAPH: capture stream and executable graphs
    cudaEvent_t ph0 = nullptr, ph1 = nullptr;  // profile: events around one phase's kernels
};

// Profile mode (params.profile = 1): CUDA events on the call's stream around the kernels of
// one phase (bin, gather, fuse); stop() waits for the end event and returns the phase's
// device time in ms.  Without profiling it records nothing and returns 0.
struct PhaseTimer {
    vgp_map* m;
    cudaStream_t st;
    bool on;
    PhaseTimer(vgp_map* mm, cudaStream_t s) : m(mm), st(s), on(mm->prm.profile != 0) {
        if (on && !m->ph0 &&
            (cudaEventCreate(&m->ph0) != cudaSuccess || cudaEventCreate(&m->ph1) != cudaSuccess)) {
            cudaGetLastError();
            on = false;
        }
        if (on) cudaEventRecord(m->ph0, st);
    }
    double stop() {
        if (!on) return 0.0;
        float ms = 0.f;
        if (cudaEventRecord(m->ph1, st) != cudaSuccess || cudaEventSynchronize(m->ph1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, m->ph0, m->ph1) != cudaSuccess) {
            cudaGetLastError();
            return 0.0;
        }
        return ms;
    }
};

struct vgp_frame {
    vgp_map* m = nullptr;
    cudaStream_t st = nullptr;
    int64_t nl = 0, T = 0, ntest = 0;
    uint64_t* leaf_key = nullptr;
    int32_t* nocc = nullptr;
    int64_t* inst_off = nullptr;
    double* X = nullptr;
    double* Xl = nullptr;
    float* Xf = nullptr;
    char4* Xi = nullptr;
    double* centre = nullptr;
    double* alpha = nullptr;
    int nprop = 0;
    double* c = nullptr;  // [ntest][nprop] surface-property means (Eq. 6)
    double* w = nullptr;  // [ntest] their variances
    uint64_t* tkey = nullptr;
    double* d = nullptr;
    double* v = nullptr;
    double* grad = nullptr;
    uint8_t* status = nullptr;
    std::vector<void*> owned;
    template <typename T_>
    T_* alloc(int64_t n, cudaStream_t s) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<int64_t>(n, 1) * sizeof(T_), s) != cudaSuccess) return nullptr;
        owned.push_back(p);
        return (T_*)p;
    }
};

static DevParams expand(const vgp_params& p) {
    DevParams P{};
    P.vs = p.voxel_size;
    P.l = p.lengthscale;
    P.l2 = p.lengthscale * p.lengthscale;
    P.inv2l2 = 1.0 / (2.0 * P.l2);
    P.s2 = p.sigma_occ * p.sigma_occ;
    P.d_max = p.d_max;
    P.log_floor = -(p.d_max * p.d_max) / (2.0 * P.l2);
    P.d_var_floor = p.d_var_floor;
    P.inv2l2_log2e = (float)(1.4426950408889634 / (2.0 * P.l2));
    P.inv2l2_hi = (float)P.inv2l2;
    P.inv2l2_lo = (float)(P.inv2l2 - (double)P.inv2l2_hi);
    P.cap_leaf = p.max_pts_leaf;
    P.cap_group = p.max_pts_group;
    P.n_props = p.n_props;
    P.emulate = p.emulate_fp64;
    P.s2p = p.sigma_prop * p.sigma_prop;
    P.search_r = p.max_leaf_search;
    P.fusion = p.fusion;
    P.precision = p.precision;
    return P;
}

static int read_words(vgp_map* m, cudaStream_t st) {
    CUDA_TRY(cudaMemcpyAsync(m->host_words, m->dev_words, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return VGP_OK;
}

static int check_err(vgp_map* m, const char* where) {
    int e = m->host_words[0];
    if (e & kErrTableFull) return fail(VGP_ERR_TABLE_FULL, "%s: hash table full", where);
    if (e & kErrTimeout) return fail(VGP_ERR_TIMEOUT, "%s: device loop limit reached", where);
    if (e & kErrCapacity) return fail(VGP_ERR_OOM, "%s: internal buffer bound exceeded", where);
    if (e & kErrAlloc) return fail(VGP_ERR_OOM, "%s: device allocation of a solve workspace failed", where);
    if (e & kErrLaunch) return fail(VGP_ERR_CUDA, "%s: CUDA graph capture, instantiation or launch failed", where);
    return VGP_OK;
}

// The ABI error code of a solve_batch return value.
static int solve_status(int rc, const char* where) {
    if (rc == 0) return VGP_OK;
    if (rc == -2) return fail(VGP_ERR_OOM, "%s: device allocation of a solve workspace failed", where);
    return fail(VGP_ERR_CUDA, "%s: CUDA graph capture, instantiation or launch failed", where);
}

#define TRY(expr)                 \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != VGP_OK) return rc_; \
    } while (0)

#define ARENA(var, type, slot, count)                                                       \
    type* var = (type*)m->ar.get(Arena::slot, sizeof(type) * (size_t)std::max<int64_t>((count), 1), st); \
    if (!var) return fail(VGP_ERR_OOM, "device allocation of %s failed", #var)

// --------------------------------------------------------------------------------------
// C ABI
// --------------------------------------------------------------------------------------
extern "C" {

const char* vgp_last_error(void) { return g_last_error.c_str(); }

int64_t vgp_launch_count(void) { return g_launches.load(); }

void vgp_default_params(vgp_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->voxel_size = 0.1;
    p->lengthscale = 0.3;
    p->sigma_occ = 0.01;
    p->d_max = 10.0;
    p->d_var_floor = 1e-3;
    p->max_pts_leaf = 64;
    p->max_pts_group = 1024;
    p->max_leaf_search = 8;
    p->fusion = VGP_FUSE_INVVAR;
    p->precision = VGP_MIXED;
    p->normal_steps = 3;
    p->sigma_prop = 0.1;
    p->n_props = 0;
}

int vgp_create(const vgp_params* p, vgp_map** out) {
    if (!p || !out) return fail(VGP_ERR_ARG, "vgp_create: null argument");
    *out = nullptr;
    if (!(p->voxel_size > 0) || !std::isfinite(p->voxel_size)) return fail(VGP_ERR_ARG, "voxel_size must be > 0");
    if (!(p->lengthscale > 0) || !std::isfinite(p->lengthscale)) return fail(VGP_ERR_ARG, "lengthscale must be > 0");
    if (!(p->sigma_occ > 0) || !std::isfinite(p->sigma_occ)) return fail(VGP_ERR_ARG, "sigma_occ must be > 0");
    if (!(p->d_max > 0) || !(p->d_var_floor > 0)) return fail(VGP_ERR_ARG, "d_max and d_var_floor must be > 0");
    if (p->max_pts_leaf < 1 || p->max_pts_leaf > 512) return fail(VGP_ERR_ARG, "max_pts_leaf must be in [1, 512]");
    if (p->max_pts_group < 1 || p->max_pts_group > 1024) return fail(VGP_ERR_ARG, "max_pts_group must be in [1, 1024]");
    if (p->max_leaf_search < 0 || p->max_leaf_search > 16) return fail(VGP_ERR_ARG, "max_leaf_search must be in [0, 16]");
    if (p->fusion != VGP_FUSE_INVVAR && p->fusion != VGP_FUSE_TSDF) return fail(VGP_ERR_ARG, "unknown fusion rule");
    if (p->precision != VGP_FP64 && p->precision != VGP_MIXED) return fail(VGP_ERR_ARG, "unknown precision");
    if (p->normal_steps < 0 || p->normal_steps > 16) return fail(VGP_ERR_ARG, "normal_steps must be in [0, 16]");
    if (p->n_props < 0 || p->n_props > 4) return fail(VGP_ERR_ARG, "n_props must be in [0, 4]");
    if (p->emulate_fp64 != 0 && p->emulate_fp64 != 1) return fail(VGP_ERR_ARG, "emulate_fp64 must be 0 or 1");
    if (!(p->sigma_prop > 0) || !std::isfinite(p->sigma_prop)) return fail(VGP_ERR_ARG, "sigma_prop must be > 0");
    if (p->launch != VGP_LAUNCH_BATCHED && p->launch != VGP_LAUNCH_PER_INSTANCE && p->launch != VGP_LAUNCH_GRAPH)
        return fail(VGP_ERR_ARG, "unknown launch mode");
    if (p->profile != 0 && p->profile != 1) return fail(VGP_ERR_ARG, "profile must be 0 or 1");
    vgp_map* m = new (std::nothrow) vgp_map();
    if (!m) return fail(VGP_ERR_OOM, "host allocation failed");
    m->prm = *p;
    m->P = expand(*p);
    cudaGetDevice(&m->device);
    if (cudaMalloc(&m->dev_words, sizeof(int) * 8) != cudaSuccess ||
        cudaMallocHost(&m->host_words, sizeof(int) * 8) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return fail(VGP_ERR_CUDA, "vgp_create: device allocation failed (is a CUDA device present?)");
    }
    cudaMemset(m->dev_words, 0, sizeof(int) * 8);
    // constant tables, computed on the host in extended precision and rounded once:
    // 2^(j/256) for the FP64 exponential, exp(-m vs^2 / (2 l^2)) for voxel-lattice distances
    std::vector<double> tab(256 + kLatticeTable);
    std::vector<float> tabf(kLatticeTable);
    for (int j = 0; j < 256; ++j) tab[j] = (double)exp2l((long double)j / 256.0L);
    const long double vs = p->voxel_size, l = p->lengthscale;
    for (int m2 = 0; m2 < kLatticeTable; ++m2) {
        const long double v = expl(-(long double)m2 * vs * vs / (2.0L * l * l));
        tab[256 + m2] = (double)v;
        tabf[m2] = (float)v;
    }
    if (cudaMalloc(&m->tables, sizeof(double) * tab.size()) != cudaSuccess ||
        cudaMalloc(&m->tables_f, sizeof(float) * tabf.size()) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(m->dev_words);
        cudaFreeHost(m->host_words);
        cudaFree(m->tables);
        delete m;
        return fail(VGP_ERR_OOM, "vgp_create: table allocation failed");
    }
    cudaMemcpy(m->tables, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(m->tables_f, tabf.data(), sizeof(float) * tabf.size(), cudaMemcpyHostToDevice);
    m->P.exp_tab = m->tables;
    m->P.lat_tab = m->tables + 256;
    m->P.lat_tab_f = m->tables_f;
    std::vector<uint8_t> mc(256 * 17, 0);
    build_mc_table(mc.data(), mc.data() + 256 * 16);
    if (cudaMalloc(&m->mc_tab, mc.size()) != cudaSuccess) {
        cudaGetLastError();
        vgp_destroy(m);
        return fail(VGP_ERR_OOM, "vgp_create: table allocation failed");
    }
    cudaMemcpy(m->mc_tab, mc.data(), mc.size(), cudaMemcpyHostToDevice);
    *out = m;
    return VGP_OK;
}

int vgp_destroy(vgp_map* m) {
    if (!m) return VGP_OK;
    cudaDeviceSynchronize();
    cudaFree(m->dev_words);
    cudaFreeHost(m->host_words);
    cudaFree(m->tables);
    cudaFree(m->tables_f);
    cudaFree(m->g.keys);
    cudaFree(m->g_slot2pool);
    cudaFree(m->g_known);
    cudaFree(m->g_D);
    cudaFree(m->g_V);
    cudaFree(m->g_flags);
    cudaFree(m->g_C);
    cudaFree(m->g_W);
    cudaFree(m->s_pts);
    cudaFree(m->s_tab.keys);
    cudaFree(m->s_slot2leaf);
    cudaFree(m->s_off);
    cudaFree(m->s_idx);
    cudaFree(m->ps_pts);
    cudaFree(m->ps_tmp);
    cudaFree(m->mc_tab);
    graph_cache_destroy(m->gcache);
    if (m->ph0) cudaEventDestroy(m->ph0);
    if (m->ph1) cudaEventDestroy(m->ph1);
    delete m;
    return VGP_OK;
}

int vgp_sync(vgp_map* m) {
    if (!m) return fail(VGP_ERR_ARG, "null map");
    CUDA_TRY(cudaDeviceSynchronize());
    return VGP_OK;
}

int vgp_get_stats(const vgp_map* m, vgp_stats* out) {
    if (!m || !out) return fail(VGP_ERR_ARG, "null argument");
    *out = m->stats;
    out->graph_replays = m->gcache.replays;
    out->graph_instantiations = m->gcache.instantiations;
    return VGP_OK;
}

// ---------------------------------- frame ----------------------------------------------
int vgp_build_frame(vgp_map* m, const float* pts, int64_t n, const double* origin, vgp_stream stream,
                    vgp_frame** out) {
    return vgp_build_frame_props(m, pts, nullptr, n, origin, stream, out);
}

int vgp_build_frame_props(vgp_map* m, const float* pts, const float* props, int64_t n, const double* origin,
                          vgp_stream stream, vgp_frame** out) {
    if (!m || !out || n < 0 || (n > 0 && !pts)) return fail(VGP_ERR_ARG, "vgp_build_frame: bad argument");
    if (props && m->prm.n_props == 0) return fail(VGP_ERR_ARG, "vgp_build_frame_props: the map has n_props = 0");
    if (n > (1ll << 30)) return fail(VGP_ERR_ARG, "vgp_build_frame: n too large");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    const DevParams& P = m->P;
    vgp_stats S{};
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 8, st));
    // 1. voxelise into the frame's leaf table
    Table ft;
    uint32_t Cf = pow2_at_least(2 * std::max<int64_t>(n, 1));
    ft.mask = Cf - 1;
    ARENA(fkeys, uint64_t, kTmp0, Cf);
    ARENA(fmasks, unsigned long long, kTmp1, (int64_t)Cf * 8);
    ARENA(fslot2leaf, int32_t, kTmp2, Cf);
    ARENA(flist, int32_t, kTmp3, Cf);
    ARENA(flkeys, uint64_t, kTmp4, Cf);
    ft.keys = fkeys;
    CUDA_TRY(cudaMemsetAsync(fkeys, 0xFF, sizeof(uint64_t) * Cf, st));
    CUDA_TRY(cudaMemsetAsync(fmasks, 0, sizeof(unsigned long long) * Cf * 8, st));
    PhaseTimer pbin(m, st);
    frame_voxelise(pts, n, P, ft, fmasks, m->dev_words + 1, m->dev_words, st);
    S.t_bin_ms = pbin.stop();
    collect_table(ft, fslot2leaf, flist, flkeys, m->dev_words + 2, Cf, m->dev_words, st);
    TRY(read_words(m, st));
    TRY(check_err(m, "vgp_build_frame"));
    const int nl = m->host_words[2];
    S.n_points = m->host_words[1];
    vgp_frame* f = new (std::nothrow) vgp_frame();
    if (!f) return fail(VGP_ERR_OOM, "host allocation failed");
    f->m = m;
    f->st = st;
    f->nl = nl;
    auto bail = [&](int code, const char* what) {
        vgp_frame_destroy(f);
        return fail(code, "vgp_build_frame: %s", what);
    };
    f->leaf_key = f->alloc<uint64_t>(nl, st);
    f->nocc = f->alloc<int32_t>(nl, st);
    f->inst_off = f->alloc<int64_t>(nl + 1, st);
    int64_t* ninst = (int64_t*)m->ar.get(Arena::kTmp5, sizeof(int64_t) * (nl + 1), st);
    if (!f->leaf_key || !f->nocc || !f->inst_off || !ninst) return bail(VGP_ERR_OOM, "allocation failed");
    if (nl > 0) cudaMemcpyAsync(f->leaf_key, flkeys, sizeof(uint64_t) * nl, cudaMemcpyDeviceToDevice, st);
    // 2. per-leaf counts, capped training sets
    frame_leaf_counts(flist, nl, fmasks, P.cap_leaf, f->nocc, ninst, st);
    exclusive_scan_i64(ninst, f->inst_off, nl, st, m->ar);
    int64_t T = 0;
    cudaMemcpyAsync(&T, f->inst_off + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return bail(VGP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    f->T = T;
    f->X = f->alloc<double>(3 * T, st);
    f->Xl = f->alloc<double>(3 * T, st);
    f->Xf = f->alloc<float>(3 * T, st);
    f->Xi = f->alloc<char4>(T, st);
    f->alpha = f->alloc<double>(T, st);
    f->centre = f->alloc<double>(3 * (int64_t)nl, st);
    if (!f->X || !f->Xl || !f->Xf || !f->Xi || !f->alpha || !f->centre) return bail(VGP_ERR_OOM, "allocation failed");
    frame_leaf_points(flist, flkeys, nl, fmasks, f->nocc, f->inst_off, P, f->X, f->Xl, f->Xf, f->Xi, f->centre, st);
    int64_t n_assigned = -1;      // ray-cast path: testing voxels with a GP node (the rest follow)
    int8_t* gsign = nullptr;
    int64_t* q_off = nullptr;
    if (!origin) {
        // 3. testing leaves: occupied leaves and their 26 neighbours
        Table tt;
        uint32_t Ct = pow2_at_least(2 * 27 * (int64_t)std::max(nl, 1));
        tt.mask = Ct - 1;
        tt.keys = (uint64_t*)m->ar.get(Arena::kTmp6, sizeof(uint64_t) * Ct, st);
        uint64_t* tl_keys = (uint64_t*)m->ar.get(Arena::kTmp7, sizeof(uint64_t) * Ct, st);
        if (!tt.keys || !tl_keys) return bail(VGP_ERR_OOM, "allocation failed");
        cudaMemsetAsync(tt.keys, 0xFF, sizeof(uint64_t) * Ct, st);
        frame_dilate(f->leaf_key, nl, tt, m->dev_words, st);
        collect_table(tt, nullptr, nullptr, tl_keys, m->dev_words + 2, Ct, m->dev_words, st);
        if (read_words(m, st) != VGP_OK) return bail(VGP_ERR_CUDA, "sync failed");
        if (check_err(m, "vgp_build_frame") != VGP_OK) {
            std::string msg = g_last_error;
            vgp_frame_destroy(f);
            g_last_error = msg;
            return VGP_ERR_TABLE_FULL;
        }
        const int ntl = m->host_words[2];
        // 4. closest-node choice per testing voxel; group voxels by instance
        int64_t* inst_cnt = (int64_t*)m->ar.get(Arena::kTmp8, sizeof(int64_t) * (nl + 1), st);
        q_off = (int64_t*)m->ar.get(Arena::kTmp9, sizeof(int64_t) * (nl + 1), st);
        int64_t* cursor = (int64_t*)m->ar.get(Arena::kTmp10, sizeof(int64_t) * (nl + 1), st);
        if (!inst_cnt || !q_off || !cursor) return bail(VGP_ERR_OOM, "allocation failed");
        cudaMemsetAsync(inst_cnt, 0, sizeof(int64_t) * (nl + 1), st);
        cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (nl + 1), st);
        frame_assign_tests(tl_keys, ntl, ft, fslot2leaf, inst_cnt, m->dev_words + 4, st);
        exclusive_scan_i64(inst_cnt, q_off, nl, st, m->ar);
        const int64_t ntest = (int64_t)ntl * 512;
        f->ntest = ntest;
        f->tkey = f->alloc<uint64_t>(ntest, st);
        f->d = f->alloc<double>(ntest, st);
        f->v = f->alloc<double>(ntest, st);
        f->grad = f->alloc<double>(3 * ntest, st);
        f->status = f->alloc<uint8_t>(ntest, st);
        if (!f->tkey || !f->d || !f->v || !f->grad || !f->status) return bail(VGP_ERR_OOM, "allocation failed");
        frame_scatter_tests(tl_keys, ntl, ft, fslot2leaf, q_off, cursor, f->tkey, st);
    } else {
        // 3'. ray-cast testing points (Sec. IV-B): surface voxels, normal voxels, known voxels on rays
        const int K = m->prm.normal_steps;
        int64_t* nocc64 = (int64_t*)m->ar.get(Arena::kTmp8, sizeof(int64_t) * (nl + 1), st);
        int64_t* soff = (int64_t*)m->ar.get(Arena::kTmp9, sizeof(int64_t) * (nl + 1), st);
        if (!nocc64 || !soff) return bail(VGP_ERR_OOM, "allocation failed");
        widen_i32(f->nocc, nocc64, nl, st);
        exclusive_scan_i64(nocc64, soff, nl, st, m->ar);
        int64_t U = 0;
        cudaMemcpyAsync(&U, soff + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return bail(VGP_ERR_CUDA, "sync failed");
        uint64_t* svox = (uint64_t*)m->ar.get(Arena::kPair0, sizeof(uint64_t) * std::max<int64_t>(U, 1), st);
        if (!svox) return bail(VGP_ERR_OOM, "allocation failed");
        frame_surface_voxels(flist, flkeys, nl, fmasks, soff, svox, st);
        double o[3] = {origin[0], origin[1], origin[2]};
        int ov[3] = {0, 0, 0}, have_o = 1;
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(o[a])) { have_o = 0; break; }
            const double t = o[a] / P.vs;
            const double u = t + 0.5;
            const double fl = std::floor(u);
            if (!(fl > -kIjkLimit && fl < kIjkLimit)) { have_o = 0; break; }
            ov[a] = (int)fl;
        }
        uint32_t Ct = pow2_at_least(2 * (U * (2 * K + 1) + (int64_t)m->g_leaves * 512 + 1024));
        Table tt;
        unsigned* tflags = nullptr;
        for (int attempt = 0;; ++attempt) {
            tt.mask = Ct - 1;
            tt.keys = (uint64_t*)m->ar.get(Arena::kTmp6, sizeof(uint64_t) * Ct, st);
            tflags = (unsigned*)m->ar.get(Arena::kTmp7, sizeof(unsigned) * Ct, st);
            if (!tt.keys || !tflags) return bail(VGP_ERR_OOM, "allocation failed");
            cudaMemsetAsync(tt.keys, 0xFF, sizeof(uint64_t) * Ct, st);
            cudaMemsetAsync(tflags, 0, sizeof(unsigned) * Ct, st);
            cudaMemsetAsync(m->dev_words, 0, sizeof(int), st);
            frame_raycast_tests(svox, U, ft, fmasks, m->g, m->g_slot2pool, m->g_known, o, have_o, ov, P.vs, K, tt, tflags,
                                m->dev_words, st);
            if (read_words(m, st) != VGP_OK) return bail(VGP_ERR_CUDA, "sync failed");
            if (!(m->host_words[0] & kErrTableFull)) break;
            if (attempt >= 4 || Ct >= (1u << 31)) return bail(VGP_ERR_TABLE_FULL, "testing-voxel table full");
            Ct <<= 2;
        }
        uint64_t* tkey_u = (uint64_t*)m->ar.get(Arena::kPair1, sizeof(uint64_t) * Ct, st);
        int8_t* tsign_u = (int8_t*)m->ar.get(Arena::kPair2, Ct, st);
        if (!tkey_u || !tsign_u) return bail(VGP_ERR_OOM, "allocation failed");
        frame_collect_tests(tt, tflags, tkey_u, tsign_u, m->dev_words + 2, st);
        if (read_words(m, st) != VGP_OK) return bail(VGP_ERR_CUDA, "sync failed");
        const int64_t nt = m->host_words[2];
        int32_t* tinst = (int32_t*)m->ar.get(Arena::kPair3, sizeof(int32_t) * std::max<int64_t>(nt, 1), st);
        int64_t* inst_cnt = (int64_t*)m->ar.get(Arena::kTmp10, sizeof(int64_t) * (nl + 1), st);
        q_off = (int64_t*)m->ar.get(Arena::kTmp15, sizeof(int64_t) * (nl + 1), st);
        int64_t* cursor = (int64_t*)m->ar.get(Arena::kTmp16, sizeof(int64_t) * (nl + 1), st);
        gsign = (int8_t*)m->ar.get(Arena::kPair4, std::max<int64_t>(nt, 1), st);
        if (!tinst || !inst_cnt || !q_off || !cursor || !gsign) return bail(VGP_ERR_OOM, "allocation failed");
        cudaMemsetAsync(inst_cnt, 0, sizeof(int64_t) * (nl + 1), st);
        cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (nl + 1), st);
        cudaMemsetAsync(m->dev_words + 4, 0, 2 * sizeof(int), st);
        frame_assign_list(tkey_u, nt, ft, fslot2leaf, P.search_r, tinst, inst_cnt, m->dev_words + 4, st);
        exclusive_scan_i64(inst_cnt, q_off, nl, st, m->ar);
        if (read_words(m, st) != VGP_OK) return bail(VGP_ERR_CUDA, "sync failed");
        n_assigned = nt - m->host_words[4];
        f->ntest = nt;
        f->tkey = f->alloc<uint64_t>(nt, st);
        f->d = f->alloc<double>(nt, st);
        f->v = f->alloc<double>(nt, st);
        f->grad = f->alloc<double>(3 * nt, st);
        f->status = f->alloc<uint8_t>(nt, st);
        if (!f->tkey || !f->d || !f->v || !f->grad || !f->status) return bail(VGP_ERR_OOM, "allocation failed");
        frame_scatter_list(tkey_u, tsign_u, nt, tinst, q_off, cursor, n_assigned, m->dev_words + 5, f->tkey, gsign, st);
        cudaMemsetAsync(m->dev_words + 4, 0, 2 * sizeof(int), st);
    }
    // 5. factorise every leaf GP and infer at its testing voxels
    SolveBatch b;
    b.n_inst = nl;
    b.inst_off = f->inst_off;
    b.Xl = f->Xl;
    b.Xf = f->Xf;
    b.Xi = f->Xi;
    b.inst_key = f->leaf_key;
    b.centre = f->centre;
    b.q_off = q_off;
    b.qkey = f->tkey;
    b.d = f->d;
    b.grad = f->grad;
    b.var = f->v;
    b.status = f->status;
    b.alpha_out = f->alpha;
    b.want_var = 1;
    SolveStats ss;
    b.max_n = P.cap_leaf;
    if (solve_batch(b, P, m->dev_words, st, m->ar, &ss, nullptr, m->prm.profile != 0, m->prm.launch, &m->cfg,
                    &m->gcache) == -2)
        return bail(VGP_ERR_OOM, "device allocation of a solve workspace failed");
    if (origin) frame_orphans_and_sign(f->ntest, n_assigned, gsign, f->d, f->grad, f->v, f->status, st);
    // 6. surface properties (Eq. 6): voxel-mean properties as targets of a second GP per leaf
    // with noise sigma_prop, inferred at the same testing voxels through the same nodes
    if (props && n > 0) {
        const int nc = m->prm.n_props;
        f->nprop = nc;
        f->c = f->alloc<double>(f->ntest * nc, st);
        f->w = f->alloc<double>(f->ntest, st);
        double* y = (double*)m->ar.get(Arena::kPair5, sizeof(double) * std::max<int64_t>(T * nc, 1), st);
        double* ycnt = (double*)m->ar.get(Arena::kPair6, sizeof(double) * std::max<int64_t>(T, 1), st);
        if (!f->c || !f->w || !y || !ycnt) return bail(VGP_ERR_OOM, "allocation failed");
        fill_u64(reinterpret_cast<uint64_t*>(f->c), 0x7ff8000000000000ull, f->ntest * nc, st);  // NaN
        fill_u64(reinterpret_cast<uint64_t*>(f->w), 0x7ff0000000000000ull, f->ntest, st);       // +inf
        cudaMemsetAsync(y, 0, sizeof(double) * T * nc, st);
        cudaMemsetAsync(ycnt, 0, sizeof(double) * T, st);
        frame_point_props(pts, props, n, nc, P, ft, fmasks, fslot2leaf, f->nocc, f->inst_off, y, ycnt, st);
        frame_prop_means(y, ycnt, T, nc, st);
        SolveBatch pb = b;
        pb.d = nullptr;
        pb.grad = nullptr;
        pb.var = nullptr;
        pb.status = nullptr;
        pb.alpha_out = nullptr;
        pb.nprop = nc;
        pb.yprop = y;
        pb.pc = f->c;
        pb.pw = f->w;
        pb.want_var = 1;
        DevParams Pp = P;
        Pp.s2 = P.s2p;
        pb.max_n = P.cap_leaf;
        if (solve_batch(pb, Pp, m->dev_words, st, m->ar, nullptr, nullptr, false, m->prm.launch, &m->cfg,
                        &m->gcache) == -2)
            return bail(VGP_ERR_OOM, "device allocation of a solve workspace failed");
    }
    if (read_words(m, st) != VGP_OK) return bail(VGP_ERR_CUDA, "sync failed");
    if (check_err(m, "vgp_build_frame") != VGP_OK) {
        std::string msg = g_last_error;
        vgp_frame_destroy(f);
        g_last_error = msg;
        return VGP_ERR_CUDA;
    }
    if (!origin && m->host_words[4] != 0) return bail(VGP_ERR_STATE, "testing voxel without a neighbouring GP leaf");
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return bail(VGP_ERR_CUDA, cudaGetErrorString(ce));
    S.n_leaves = nl;
    S.n_instances = nl;
    S.n_train = T;
    S.n_queries = f->ntest;
    for (int i = 0; i < 5; ++i) S.bucket_count[i] = ss.bucket_count[i];
    S.sum_n3 = ss.sum_n3;
    S.sum_n2 = ss.sum_n2;
    S.t_solve_ms = ss.t_solve_ms;
    for (int i = 0; i < 5; ++i) {
        S.t_bucket_ms[i] = ss.t_bucket_ms[i];
        S.cfg_threads[i] = m->cfg.threads[i];
        S.cfg_per_sm[i] = m->cfg.per_sm[i];
    }
    S.cfg_stage_panel = m->cfg.stage_panel;
    S.graph_replays = m->gcache.replays;
    S.graph_instantiations = m->gcache.instantiations;
    S.grid_leaves = m->g_leaves;
    S.grid_capacity_leaves = m->pool_cap;
    m->stats = S;
    *out = f;
    return VGP_OK;
}

int vgp_frame_results(const vgp_frame* f, int64_t* n_test, const uint64_t** keys, const double** d,
                      const double** v, const double** grad, const uint8_t** status) {
    if (!f) return fail(VGP_ERR_ARG, "null frame");
    if (n_test) *n_test = f->ntest;
    if (keys) *keys = f->tkey;
    if (d) *d = f->d;
    if (v) *v = f->v;
    if (grad) *grad = f->grad;
    if (status) *status = f->status;
    return VGP_OK;
}

int vgp_frame_props(const vgp_frame* f, int32_t* n_props, const double** c, const double** w) {
    if (!f) return fail(VGP_ERR_ARG, "null frame");
    if (n_props) *n_props = f->nprop;
    if (c) *c = f->c;
    if (w) *w = f->w;
    return VGP_OK;
}

int vgp_frame_instances(const vgp_frame* f, int64_t* n_leaves, int64_t* n_train, const uint64_t** leaf_key,
                        const int32_t** n_occ, const int64_t** inst_off, const double** X, const double** alpha) {
    if (!f) return fail(VGP_ERR_ARG, "null frame");
    if (n_leaves) *n_leaves = f->nl;
    if (n_train) *n_train = f->T;
    if (leaf_key) *leaf_key = f->leaf_key;
    if (n_occ) *n_occ = f->nocc;
    if (inst_off) *inst_off = f->inst_off;
    if (X) *X = f->X;
    if (alpha) *alpha = f->alpha;
    return VGP_OK;
}

int vgp_frame_destroy(vgp_frame* f) {
    if (!f) return VGP_OK;
    for (void* p : f->owned) cudaFreeAsync(p, f->st);
    cudaStreamSynchronize(f->st);
    delete f;
    return VGP_OK;
}

// ---------------------------------- fusion ---------------------------------------------
static PropGrid prop_grid(const vgp_map* m) {
    PropGrid pg;
    if (m->prm.n_props > 0 && m->g_C) {
        pg.C = m->g_C;
        pg.W = m->g_W;
        pg.nc = m->prm.n_props;
    }
    return pg;
}

static int grid_reserve(vgp_map* m, int64_t extra_leaves, cudaStream_t st) {
    const int64_t need = m->g_leaves + extra_leaves;
    if (need > (1ll << 30)) return fail(VGP_ERR_OOM, "grid too large");
    // payload pool
    if (need > m->pool_cap) {
        int64_t nc = std::max<int64_t>(need, std::max<int64_t>(1024, (int64_t)m->pool_cap * 2));
        unsigned long long* known = nullptr;
        double *D = nullptr, *V = nullptr;
        int32_t* flags = nullptr;
        if (cudaMalloc(&known, sizeof(unsigned long long) * 8 * nc) != cudaSuccess ||
            cudaMalloc(&D, sizeof(double) * 512 * nc) != cudaSuccess ||
            cudaMalloc(&V, sizeof(double) * 512 * nc) != cudaSuccess ||
            cudaMalloc(&flags, sizeof(int32_t) * nc) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(known); cudaFree(D); cudaFree(V); cudaFree(flags);
            return fail(VGP_ERR_OOM, "grid pool allocation failed (%lld leaves)", (long long)nc);
        }
        if (m->g_leaves > 0) {
            cudaMemcpyAsync(known, m->g_known, sizeof(unsigned long long) * 8 * m->g_leaves, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(D, m->g_D, sizeof(double) * 512 * m->g_leaves, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(V, m->g_V, sizeof(double) * 512 * m->g_leaves, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(flags, m->g_flags, sizeof(int32_t) * m->g_leaves, cudaMemcpyDeviceToDevice, st);
        }
        const int np = m->prm.n_props;
        double *Cp = nullptr, *Wp = nullptr;
        if (np > 0) {
            if (cudaMalloc(&Cp, sizeof(double) * 512 * np * nc) != cudaSuccess ||
                cudaMalloc(&Wp, sizeof(double) * 512 * nc) != cudaSuccess) {
                cudaGetLastError();
                cudaStreamSynchronize(st);
                cudaFree(known); cudaFree(D); cudaFree(V); cudaFree(flags); cudaFree(Cp); cudaFree(Wp);
                return fail(VGP_ERR_OOM, "grid property pool allocation failed (%lld leaves)", (long long)nc);
            }
            if (m->g_leaves > 0) {
                cudaMemcpyAsync(Cp, m->g_C, sizeof(double) * 512 * np * m->g_leaves, cudaMemcpyDeviceToDevice, st);
                cudaMemcpyAsync(Wp, m->g_W, sizeof(double) * 512 * m->g_leaves, cudaMemcpyDeviceToDevice, st);
            }
        }
        CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(m->g_known); cudaFree(m->g_D); cudaFree(m->g_V); cudaFree(m->g_flags);
        cudaFree(m->g_C); cudaFree(m->g_W);
        m->g_known = known; m->g_D = D; m->g_V = V; m->g_flags = flags;
        m->g_C = Cp; m->g_W = Wp;
        m->pool_cap = (int)nc;
    }
    // hash table at load <= 1/2
    if ((int64_t)m->g.cap() < 2 * need) {
        Table nt;
        uint32_t cap = pow2_at_least(std::max<int64_t>(4 * need, 1024));
        nt.mask = cap - 1;
        int32_t* ns2p = nullptr;
        if (cudaMalloc(&nt.keys, sizeof(uint64_t) * cap) != cudaSuccess ||
            cudaMalloc(&ns2p, sizeof(int32_t) * cap) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(nt.keys); cudaFree(ns2p);
            return fail(VGP_ERR_OOM, "grid table allocation failed");
        }
        cudaMemsetAsync(nt.keys, 0xFF, sizeof(uint64_t) * cap, st);
        cudaMemsetAsync(ns2p, 0xFF, sizeof(int32_t) * cap, st);
        if (m->g.keys) grid_rehash(m->g, m->g_slot2pool, nt, ns2p, m->dev_words, st);
        CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(m->g.keys); cudaFree(m->g_slot2pool);
        m->g = nt;
        m->g_slot2pool = ns2p;
    }
    return VGP_OK;
}

int vgp_fuse(vgp_map* m, vgp_frame* f, vgp_stream stream) {
    if (!m || !f || f->m != m) return fail(VGP_ERR_ARG, "vgp_fuse: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 3, st));
    TRY(grid_reserve(m, f->ntest / 512 + 1, st));
    CUDA_TRY(cudaMemcpyAsync(m->dev_words + 3, &m->g_leaves, sizeof(int), cudaMemcpyHostToDevice, st));
    PhaseTimer pfuse(m, st);
    fuse_clear_flags(m->g_flags, m->g_leaves, st);
    fuse_insert(f->tkey, f->d, f->v, f->status, f->ntest, m->prm.fusion, m->g, m->g_slot2pool, m->dev_words, st);
    const PropGrid pg = prop_grid(m);
    PropIn pin;
    if (pg.nc > 0 && f->nprop == pg.nc) {
        pin.c = f->c;
        pin.w = f->w;
        pin.nc = f->nprop;
    }
    fuse_alloc(m->g_slot2pool, m->g, m->dev_words + 3, m->pool_cap, m->g_known, m->g_flags, m->dev_words, pg, st);
    fuse_update(f->tkey, f->d, f->v, f->status, f->ntest, m->prm.fusion, m->g, m->g_slot2pool, m->g_known, m->g_D,
                m->g_V, m->g_flags, pin, pg, st);
    const double t_fuse = pfuse.stop();
    TRY(read_words(m, st));
    TRY(check_err(m, "vgp_fuse"));
    m->stats.t_fuse_ms = t_fuse;
    CUDA_TRY(cudaGetLastError());
    m->g_leaves = m->host_words[3];
    m->stats.grid_leaves = m->g_leaves;
    m->stats.grid_capacity_leaves = m->pool_cap;
    return VGP_OK;
}

int vgp_export_grid(vgp_map* m, int64_t* n, uint64_t* keys, double* D, double* V, uint8_t* flags, vgp_stream stream) {
    if (!m || !n) return fail(VGP_ERR_ARG, "vgp_export_grid: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t cap_out = (int64_t)m->g_leaves * 512;
    if (m->g_leaves == 0) {
        *n = 0;
        return VGP_OK;
    }
    ARENA(okey, uint64_t, kTmp0, cap_out);
    ARENA(oD, double, kTmp1, cap_out);
    ARENA(oV, double, kTmp2, cap_out);
    ARENA(ofl, uint8_t, kTmp3, cap_out);
    grid_export(m->g, m->g_slot2pool, m->g_known, m->g_D, m->g_V, m->g_flags, m->dev_words + 2, okey, oD, oV, ofl, st);
    TRY(read_words(m, st));
    const int64_t cnt = m->host_words[2];
    if (!keys) {
        *n = cnt;
        return VGP_OK;
    }
    if (*n < cnt) return fail(VGP_ERR_ARG, "vgp_export_grid: arrays hold %lld < %lld", (long long)*n, (long long)cnt);
    std::vector<uint64_t> hk(cnt);
    std::vector<double> hD(cnt), hV(cnt);
    std::vector<uint8_t> hf(cnt);
    CUDA_TRY(cudaMemcpyAsync(hk.data(), okey, sizeof(uint64_t) * cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hD.data(), oD, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hV.data(), oV, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hf.data(), ofl, cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> ord(cnt);
    for (int64_t i = 0; i < cnt; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return hk[a] < hk[b]; });
    for (int64_t i = 0; i < cnt; ++i) {
        keys[i] = hk[ord[i]];
        if (D) D[i] = hD[ord[i]];
        if (V) V[i] = hV[ord[i]];
        if (flags) flags[i] = hf[ord[i]];
    }
    *n = cnt;
    return VGP_OK;
}

int vgp_import_grid(vgp_map* m, int64_t n, const uint64_t* keys, const double* D, const double* V,
                    const uint8_t* flags, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!keys || !D || !V || !flags))) return fail(VGP_ERR_ARG, "vgp_import_grid: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    // clear the current grid
    if (m->g.keys) {
        CUDA_TRY(cudaMemsetAsync(m->g.keys, 0xFF, sizeof(uint64_t) * m->g.cap(), st));
        CUDA_TRY(cudaMemsetAsync(m->g_slot2pool, 0xFF, sizeof(int32_t) * m->g.cap(), st));
    }
    m->g_leaves = 0;
    if (n == 0) return VGP_OK;
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 8, st));
    TRY(grid_reserve(m, n, st));  // at most one leaf per voxel
    ARENA(ik, uint64_t, kTmp0, n);
    ARENA(iD, double, kTmp1, n);
    ARENA(iV, double, kTmp2, n);
    ARENA(ifl, uint8_t, kTmp3, n);
    CUDA_TRY(cudaMemcpyAsync(ik, keys, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(iD, D, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(iV, V, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(ifl, flags, n, cudaMemcpyHostToDevice, st));
    grid_import(ik, iD, iV, ifl, n, m->g, m->g_slot2pool, m->dev_words + 3, m->pool_cap, m->g_known, m->g_D, m->g_V,
                m->g_flags, m->dev_words, prop_grid(m), st);
    TRY(read_words(m, st));
    TRY(check_err(m, "vgp_import_grid"));
    m->g_leaves = m->host_words[3];
    return VGP_OK;
}

int vgp_export_props(vgp_map* m, int64_t* n, uint64_t* keys, double* C, double* W, vgp_stream stream) {
    if (!m || !n) return fail(VGP_ERR_ARG, "vgp_export_props: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const PropGrid pg = prop_grid(m);
    if (m->g_leaves == 0 || pg.nc == 0) {
        *n = 0;
        return VGP_OK;
    }
    const int64_t cap_out = (int64_t)m->g_leaves * 512;
    ARENA(okey, uint64_t, kTmp0, cap_out);
    ARENA(oC, double, kTmp1, cap_out * pg.nc);
    ARENA(oW, double, kTmp2, cap_out);
    grid_export_props(m->g, m->g_slot2pool, m->g_known, pg, m->dev_words + 2, okey, oC, oW, st);
    TRY(read_words(m, st));
    const int64_t cnt = m->host_words[2];
    if (!keys) {
        *n = cnt;
        return VGP_OK;
    }
    if (*n < cnt) return fail(VGP_ERR_ARG, "vgp_export_props: arrays hold %lld < %lld", (long long)*n, (long long)cnt);
    std::vector<uint64_t> hk(cnt);
    std::vector<double> hC(cnt * pg.nc), hW(cnt);
    CUDA_TRY(cudaMemcpyAsync(hk.data(), okey, sizeof(uint64_t) * cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hC.data(), oC, sizeof(double) * cnt * pg.nc, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hW.data(), oW, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> ord(cnt);
    for (int64_t i = 0; i < cnt; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return hk[a] < hk[b]; });
    for (int64_t i = 0; i < cnt; ++i) {
        keys[i] = hk[ord[i]];
        if (C)
            for (int ch = 0; ch < pg.nc; ++ch) C[i * pg.nc + ch] = hC[ord[i] * pg.nc + ch];
        if (W) W[i] = hW[ord[i]];
    }
    *n = cnt;
    return VGP_OK;
}

int vgp_import_props(vgp_map* m, int64_t n, const uint64_t* keys, const double* C, const double* W, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!keys || !C || !W))) return fail(VGP_ERR_ARG, "vgp_import_props: bad argument");
    const PropGrid pg = prop_grid(m);
    if (n == 0) return VGP_OK;
    if (pg.nc == 0) return fail(VGP_ERR_STATE, "vgp_import_props: the map holds no properties (n_props = 0 or empty grid)");
    cudaStream_t st = (cudaStream_t)stream;
    ARENA(ik, uint64_t, kTmp0, n);
    ARENA(iC, double, kTmp1, n * pg.nc);
    ARENA(iW, double, kTmp2, n);
    CUDA_TRY(cudaMemcpyAsync(ik, keys, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(iC, C, sizeof(double) * n * pg.nc, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(iW, W, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    grid_import_props(ik, iC, iW, n, m->g, m->g_slot2pool, m->g_known, pg, st);
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    return VGP_OK;
}

// ---------------------------------- surface --------------------------------------------
int vgp_set_surface(vgp_map* m, const float* pts, int64_t n, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && !pts)) return fail(VGP_ERR_ARG, "vgp_set_surface: bad argument");
    if (n >= (1ll << 31)) return fail(VGP_ERR_ARG, "vgp_set_surface: at most 2^31 - 1 points");
    cudaStream_t st = (cudaStream_t)stream;
    const DevParams& P = m->P;
    m->has_surface = false;
    if (n > m->s_pts_cap) {
        cudaFree(m->s_pts);
        m->s_pts = nullptr;
        if (cudaMalloc(&m->s_pts, sizeof(float) * 3 * n) != cudaSuccess) {
            cudaGetLastError();
            m->s_pts_cap = 0;
            return fail(VGP_ERR_OOM, "surface copy allocation failed");
        }
        m->s_pts_cap = n;
    }
    if (n > 0) CUDA_TRY(cudaMemcpyAsync(m->s_pts, pts, sizeof(float) * 3 * n, cudaMemcpyDeviceToDevice, st));
    m->s_n = n;
    uint32_t Cs = pow2_at_least(2 * std::max<int64_t>(n, 1));
    if (m->s_tab.cap() != Cs) {
        cudaFree(m->s_tab.keys);
        cudaFree(m->s_slot2leaf);
        m->s_tab.keys = nullptr;
        m->s_slot2leaf = nullptr;
        if (cudaMalloc(&m->s_tab.keys, sizeof(uint64_t) * Cs) != cudaSuccess ||
            cudaMalloc(&m->s_slot2leaf, sizeof(int32_t) * Cs) != cudaSuccess) {
            cudaGetLastError();
            return fail(VGP_ERR_OOM, "surface table allocation failed");
        }
        m->s_tab.mask = Cs - 1;
    }
    CUDA_TRY(cudaMemsetAsync(m->s_tab.keys, 0xFF, sizeof(uint64_t) * Cs, st));
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 8, st));
    ARENA(pt_slot, int32_t, kTmp0, n);
    ARENA(slot_cnt, int32_t, kTmp1, Cs);
    ARENA(list, int32_t, kTmp2, Cs);
    CUDA_TRY(cudaMemsetAsync(slot_cnt, 0, sizeof(int32_t) * Cs, st));
    PhaseTimer pbin(m, st);
    surface_bin(m->s_pts, n, P, m->s_tab, pt_slot, slot_cnt, m->dev_words + 1, m->dev_words, st);
    const double t_bin = pbin.stop();
    collect_table(m->s_tab, m->s_slot2leaf, list, nullptr, m->dev_words + 2, Cs, m->dev_words, st);
    TRY(read_words(m, st));
    TRY(check_err(m, "vgp_set_surface"));
    const int nl = m->host_words[2];
    m->stats = vgp_stats{};
    m->stats.t_bin_ms = t_bin;
    m->stats.n_points = m->host_words[1];
    m->stats.n_leaves = nl;
    if (nl + 1 > m->s_off_cap) {
        cudaFree(m->s_off);
        if (cudaMalloc(&m->s_off, sizeof(int64_t) * (nl + 1)) != cudaSuccess) {
            cudaGetLastError();
            m->s_off = nullptr;
            m->s_off_cap = 0;
            return fail(VGP_ERR_OOM, "surface offsets allocation failed");
        }
        m->s_off_cap = nl + 1;
    }
    const int64_t nv = m->host_words[1];
    if (nv > m->s_idx_cap) {
        cudaFree(m->s_idx);
        if (cudaMalloc(&m->s_idx, sizeof(int32_t) * std::max<int64_t>(nv, 1)) != cudaSuccess) {
            cudaGetLastError();
            m->s_idx = nullptr;
            m->s_idx_cap = 0;
            return fail(VGP_ERR_OOM, "surface index allocation failed");
        }
        m->s_idx_cap = nv;
    }
    ARENA(cnt, int64_t, kTmp3, nl + 1);
    ARENA(cursor, int32_t, kTmp4, nl + 1);
    surface_leaf_counts(list, nl, slot_cnt, cnt, st);
    exclusive_scan_i64(cnt, m->s_off, nl, st, m->ar);
    CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (nl + 1), st));
    surface_scatter(pt_slot, n, m->s_slot2leaf, m->s_off, cursor, m->s_idx, nl, st);
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    m->s_nl = nl;
    m->has_surface = true;
    return VGP_OK;
}

// ------------------------- zero crossings and marching cubes (Sec. IV-D) ----------------
static GridView grid_view(const vgp_map* m) {
    GridView g{m->g.keys, m->g.mask, m->g_slot2pool, m->g_known, m->g_D};
    const PropGrid pg = prop_grid(m);
    g.C = pg.C;
    g.W = pg.W;
    g.nc = pg.nc;
    return g;
}

// leaves of the grid (all, or those the latest fusion touched), in arena slots kTmp5/kTmp6
static int select_leaves(vgp_map* m, int active_only, cudaStream_t st, int32_t** lpool, uint64_t** lkey, int* nl) {
    *nl = 0;
    if (!m->g.keys || m->g_leaves <= 0) return VGP_OK;
    ARENA(lp, int32_t, kTmp5, m->g_leaves);
    ARENA(lk, uint64_t, kTmp6, m->g_leaves);
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 8, st));
    mesh_leaf_list(grid_view(m), m->g_flags, active_only, lp, lk, m->dev_words + 2, st);
    TRY(read_words(m, st));
    *nl = m->host_words[2];
    *lpool = lp;
    *lkey = lk;
    return VGP_OK;
}

// the last entry of a device offset array
static int read_total(const int64_t* off_end, cudaStream_t st, int64_t* total) {
    CUDA_TRY(cudaMemcpyAsync(total, off_end, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return VGP_OK;
}

struct vgp_mesh {
    int64_t nx = 0, nt = 0;
    float* xyz = nullptr;
    uint64_t* owner = nullptr;
    uint8_t* slot = nullptr;
    double* txyz = nullptr;
    uint64_t* tkey = nullptr;
    uint8_t* taxis = nullptr;
    int nprop = 0;
    double* xprop = nullptr;  // [nx][nprop]
    double* tprop = nullptr;  // [nt][3][nprop]
};

void vgp_mesh_destroy(vgp_mesh* h) {
    if (!h) return;
    cudaFree(h->xyz);
    cudaFree(h->owner);
    cudaFree(h->slot);
    cudaFree(h->txyz);
    cudaFree(h->tkey);
    cudaFree(h->taxis);
    cudaFree(h->xprop);
    cudaFree(h->tprop);
    delete h;
}

static int extract_into(vgp_map* m, int active_only, int want_triangles, cudaStream_t st, vgp_mesh* h) {
    int32_t* lp = nullptr;
    uint64_t* lk = nullptr;
    int nl = 0;
    TRY(select_leaves(m, active_only, st, &lp, &lk, &nl));
    if (nl == 0) return VGP_OK;
    const double vs = m->prm.voxel_size;
    const GridView g = grid_view(m);
    ARENA(cnt, int64_t, kTmp7, nl + 1);
    ARENA(off, int64_t, kTmp8, nl + 1);
    h->nprop = g.nc;
    mesh_crossings(g, lp, lk, nl, vs, cnt, nullptr, 0, nullptr, nullptr, nullptr, nullptr, false, st);
    exclusive_scan_i64(cnt, off, nl, st, m->ar);
    TRY(read_total(off + nl, st, &h->nx));
    if (cudaMalloc(&h->xyz, sizeof(float) * 3 * std::max<int64_t>(h->nx, 1)) != cudaSuccess ||
        cudaMalloc(&h->owner, sizeof(uint64_t) * std::max<int64_t>(h->nx, 1)) != cudaSuccess ||
        cudaMalloc(&h->slot, std::max<int64_t>(h->nx, 1)) != cudaSuccess ||
        (g.nc > 0 && cudaMalloc(&h->xprop, sizeof(double) * g.nc * std::max<int64_t>(h->nx, 1)) != cudaSuccess)) {
        cudaGetLastError();
        return fail(VGP_ERR_OOM, "vgp_extract_mesh: crossing allocation failed");
    }
    mesh_crossings(g, lp, lk, nl, vs, cnt, off, 0, h->xyz, h->owner, h->slot, h->xprop, true, st);
    if (want_triangles) {
        const uint8_t* tab = m->mc_tab;
        mesh_triangles(g, lp, lk, nl, tab, tab + 256 * 16, vs, cnt, nullptr, nullptr, nullptr, nullptr, nullptr, false,
                       st);
        exclusive_scan_i64(cnt, off, nl, st, m->ar);
        TRY(read_total(off + nl, st, &h->nt));
        if (cudaMalloc(&h->txyz, sizeof(double) * 9 * std::max<int64_t>(h->nt, 1)) != cudaSuccess ||
            cudaMalloc(&h->tkey, sizeof(uint64_t) * 3 * std::max<int64_t>(h->nt, 1)) != cudaSuccess ||
            cudaMalloc(&h->taxis, 3 * std::max<int64_t>(h->nt, 1)) != cudaSuccess ||
            (g.nc > 0 && cudaMalloc(&h->tprop, sizeof(double) * 3 * g.nc * std::max<int64_t>(h->nt, 1)) != cudaSuccess)) {
            cudaGetLastError();
            return fail(VGP_ERR_OOM, "vgp_extract_mesh: triangle allocation failed");
        }
        mesh_triangles(g, lp, lk, nl, tab, tab + 256 * 16, vs, cnt, off, h->txyz, h->tkey, h->taxis, h->tprop, true,
                       st);
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    return VGP_OK;
}

int vgp_extract_mesh(vgp_map* m, int active_only, int want_triangles, vgp_stream stream, vgp_mesh** out) {
    if (!m || !out || (active_only != 0 && active_only != 1) || (want_triangles != 0 && want_triangles != 1))
        return fail(VGP_ERR_ARG, "vgp_extract_mesh: bad argument");
    *out = nullptr;
    vgp_mesh* h = new (std::nothrow) vgp_mesh();
    if (!h) return fail(VGP_ERR_OOM, "host allocation failed");
    const int rc = extract_into(m, active_only, want_triangles, (cudaStream_t)stream, h);
    if (rc != VGP_OK) {
        vgp_mesh_destroy(h);
        return rc;
    }
    *out = h;
    return VGP_OK;
}

int vgp_mesh_crossings(const vgp_mesh* h, int64_t* n, const float** xyz, const uint64_t** owner,
                       const uint8_t** slot) {
    if (!h || !n) return fail(VGP_ERR_ARG, "vgp_mesh_crossings: null argument");
    *n = h->nx;
    if (xyz) *xyz = h->xyz;
    if (owner) *owner = h->owner;
    if (slot) *slot = h->slot;
    return VGP_OK;
}

int vgp_mesh_props(const vgp_mesh* h, int32_t* n_props, const double** cross, const double** vert) {
    if (!h) return fail(VGP_ERR_ARG, "vgp_mesh_props: null mesh");
    if (n_props) *n_props = h->nprop;
    if (cross) *cross = h->xprop;
    if (vert) *vert = h->tprop;
    return VGP_OK;
}

int vgp_mesh_triangles(const vgp_mesh* h, int64_t* n, const double** xyz, const uint64_t** edge_key,
                       const uint8_t** edge_axis) {
    if (!h || !n) return fail(VGP_ERR_ARG, "vgp_mesh_triangles: null argument");
    *n = h->nt;
    if (xyz) *xyz = h->txyz;
    if (edge_key) *edge_key = h->tkey;
    if (edge_axis) *edge_axis = h->taxis;
    return VGP_OK;
}

void vgp_debug_mc_table(uint8_t* tab, uint8_t* ntri) {
    if (!tab || !ntri) return;
    std::fill(tab, tab + 256 * 16, (uint8_t)0);
    build_mc_table(tab, ntri);
}

static int grow_f32(float** p, int64_t* cap, int64_t need) {
    if (need <= *cap) return VGP_OK;
    const int64_t c = std::max<int64_t>(need + need / 4, 1024);
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, sizeof(float) * 3 * c) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(VGP_ERR_OOM, "training-set allocation failed");
    }
    *cap = c;
    return VGP_OK;
}

int vgp_update_surface(vgp_map* m, vgp_stream stream) {
    if (!m) return fail(VGP_ERR_ARG, "vgp_update_surface: null map");
    cudaStream_t st = (cudaStream_t)stream;
    const double vs = m->prm.voxel_size;
    const GridView g = grid_view(m);
    const bool have_grid = m->g.keys && m->g_leaves > 0;
    // 1. the stored points of leaves the latest fusion did not touch stay, in order
    const int64_t n0 = m->ps_n;
    int64_t kept = n0;
    int64_t* keep = nullptr;
    int64_t* pos = nullptr;
    if (n0 > 0 && have_grid) {
        ARENA(keep_, int64_t, kTmp9, n0 + 1);
        ARENA(pos_, int64_t, kTmp10, n0 + 1);
        keep = keep_;
        pos = pos_;
        store_keep(m->ps_pts, n0, vs, g, m->g_flags, keep, st);
        exclusive_scan_i64(keep, pos, n0, st, m->ar);
        TRY(read_total(pos + n0, st, &kept));
    }
    // 2. crossings of the touched leaves
    int32_t* lp = nullptr;
    uint64_t* lk = nullptr;
    int nl = 0;
    int64_t added = 0;
    int64_t *cnt = nullptr, *off = nullptr;
    if (have_grid) {
        TRY(select_leaves(m, 1, st, &lp, &lk, &nl));
        if (nl > 0) {
            ARENA(cnt_, int64_t, kTmp7, nl + 1);
            ARENA(off_, int64_t, kTmp8, nl + 1);
            cnt = cnt_;
            off = off_;
            mesh_crossings(g, lp, lk, nl, vs, cnt, nullptr, 0, nullptr, nullptr, nullptr, nullptr, false, st);
            exclusive_scan_i64(cnt, off, nl, st, m->ar);
            TRY(read_total(off + nl, st, &added));
        }
    }
    // 3. new training set = kept points, then the new crossings leaf by leaf
    const int64_t n1 = kept + added;
    if (n1 >= (1ll << 31)) return fail(VGP_ERR_ARG, "vgp_update_surface: training set above 2^31 - 1 points");
    TRY(grow_f32(&m->ps_tmp, &m->ps_tmp_cap, n1));
    if (keep)
        store_compact(m->ps_pts, n0, keep, pos, m->ps_tmp, st);
    else if (n0 > 0)
        CUDA_TRY(cudaMemcpyAsync(m->ps_tmp, m->ps_pts, sizeof(float) * 3 * n0, cudaMemcpyDeviceToDevice, st));
    if (added > 0) mesh_crossings(g, lp, lk, nl, vs, cnt, off, kept, m->ps_tmp, nullptr, nullptr, nullptr, true, st);
    std::swap(m->ps_pts, m->ps_tmp);
    std::swap(m->ps_cap, m->ps_tmp_cap);
    m->ps_n = n1;
    // 4. the G-GPDF is trained on the new set
    return vgp_set_surface(m, m->ps_pts, n1, stream);
}

int vgp_surface_points(vgp_map* m, int64_t* n, const float** xyz) {
    if (!m || !n) return fail(VGP_ERR_ARG, "vgp_surface_points: null argument");
    *n = m->ps_n;
    if (xyz) *xyz = m->ps_pts;
    return VGP_OK;
}

// ---------------------------------- queries --------------------------------------------
struct QueryPlan {
    int64_t n = 0;
    int ni = 0, ng = 0;
    int64_t T = 0;
    uint64_t* ikeys = nullptr;   // centre leaf key of each instance
    int32_t* q_inst = nullptr;   // instance of each query (< 0: none)
    double t_gather_ms = 0;      // profile: the gather kernel
    int64_t n_cand = 0;          // profile: candidate points the gather scanned
    int64_t* inst_off = nullptr;
    double* Xl = nullptr;
    float* Xf = nullptr;
    double* centre = nullptr;
    int64_t* gidx = nullptr;
    int64_t* q_off = nullptr;
    int64_t* qidx = nullptr;
};

// Query leaves (groups) of a batch and the centre leaf of each group's neighbourhood.
struct GroupPlan {
    int ng = 0;
    int32_t* q_slot = nullptr;      // per query: slot in the query-leaf table, < 0 invalid
    int32_t* slot2group = nullptr;
    uint64_t* gcen = nullptr;       // per group: centre leaf key, kEmpty if no support
};

static int plan_groups(vgp_map* m, const float* q, int64_t n, cudaStream_t st, GroupPlan& G) {
    const DevParams& P = m->P;
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 8, st));
    Table qt;
    uint32_t Cq = pow2_at_least(2 * std::min<int64_t>(std::max<int64_t>(n, 1), 1ll << 21));
    ARENA(q_slot, int32_t, kTmp0, n);
    for (int attempt = 0;; ++attempt) {
        qt.mask = Cq - 1;
        qt.keys = (uint64_t*)m->ar.get(Arena::kTmp1, sizeof(uint64_t) * Cq, st);
        if (!qt.keys) return fail(VGP_ERR_OOM, "query table allocation failed");
        CUDA_TRY(cudaMemsetAsync(qt.keys, 0xFF, sizeof(uint64_t) * Cq, st));
        CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int), st));
        query_leaf(q, n, P, qt, q_slot, m->dev_words, st);
        TRY(read_words(m, st));
        if (!(m->host_words[0] & kErrTableFull)) break;
        if (attempt >= 6 || Cq >= (1u << 31)) return fail(VGP_ERR_TABLE_FULL, "query leaf table full");
        Cq <<= 2;
    }
    ARENA(slot2group, int32_t, kTmp2, Cq);
    ARENA(gkeys, uint64_t, kTmp3, Cq);
    collect_table(qt, slot2group, nullptr, gkeys, m->dev_words + 2, Cq, m->dev_words, st);
    TRY(read_words(m, st));
    TRY(check_err(m, "query"));
    const int ng = m->host_words[2];
    ARENA(gcen, uint64_t, kTmp4, ng);
    group_centre(gkeys, ng, m->s_tab, P.search_r, gcen, st);
    G.ng = ng;
    G.q_slot = q_slot;
    G.slot2group = slot2group;
    G.gcen = gcen;
    return VGP_OK;
}

static int plan_queries(vgp_map* m, const float* q, int64_t n, double* d, double* grad, double* var, uint8_t* status,
                        cudaStream_t st, QueryPlan& Q) {
    const DevParams& P = m->P;
    Q.n = n;
    GroupPlan G;
    TRY(plan_groups(m, q, n, st, G));
    const int ng = G.ng;
    Q.ng = ng;
    int32_t* q_slot = G.q_slot;
    int32_t* slot2group = G.slot2group;
    uint64_t* gcen = G.gcen;
    // unique centres -> instances
    Table it;
    uint32_t Ci = pow2_at_least(2 * (int64_t)std::max(ng, 1));
    it.mask = Ci - 1;
    it.keys = (uint64_t*)m->ar.get(Arena::kTmp5, sizeof(uint64_t) * Ci, st);
    ARENA(islot2inst, int32_t, kTmp6, Ci);
    ARENA(ikeys, uint64_t, kTmp7, Ci);
    if (!it.keys) return fail(VGP_ERR_OOM, "instance table allocation failed");
    CUDA_TRY(cudaMemsetAsync(it.keys, 0xFF, sizeof(uint64_t) * Ci, st));
    insert_centres(gcen, ng, it, m->dev_words, st);
    collect_table(it, islot2inst, nullptr, ikeys, m->dev_words + 2, Ci, m->dev_words, st);
    TRY(read_words(m, st));
    TRY(check_err(m, "query"));
    const int ni = m->host_words[2];
    Q.ni = ni;
    ARENA(ncand, int64_t, kTmp8, ni + 1);
    ARENA(ninst, int64_t, kTmp9, ni + 1);
    ARENA(inst_off, int64_t, kTmp10, ni + 1);
    inst_count(ikeys, ni, m->s_tab, m->s_slot2leaf, m->s_off, P.cap_group, ncand, ninst, st);
    exclusive_scan_i64(ninst, inst_off, ni, st, m->ar);
    int64_t T = 0;
    CUDA_TRY(cudaMemcpyAsync(&T, inst_off + ni, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    Q.T = T;
    ARENA(Xl, double, kTmp11, 3 * T);
    ARENA(Xf, float, kTmp12, 3 * T);
    ARENA(gidx, int64_t, kTmp13, T);
    ARENA(centre, double, kTmp14, 3 * (int64_t)ni);
    if (m->prm.profile) {  // candidate count of the gather, for its algorithmic bytes
        std::vector<int64_t> hc(ni);
        if (ni) CUDA_TRY(cudaMemcpyAsync(hc.data(), ncand, sizeof(int64_t) * ni, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < ni; ++i) Q.n_cand += hc[i];
    }
    PhaseTimer pgat(m, st);
    inst_gather(ikeys, ni, m->s_tab, m->s_slot2leaf, m->s_off, m->s_idx, m->s_pts, ncand, inst_off, P, Xl, Xf, gidx,
                centre, st);
    Q.t_gather_ms = pgat.stop();
    // route queries to instances
    ARENA(q_inst, int32_t, kTmp15, n);
    ARENA(inst_qcnt, int64_t, kTmp16, ni + 1);
    ARENA(q_off, int64_t, kTmp17, ni + 1);
    CUDA_TRY(cudaMemsetAsync(inst_qcnt, 0, sizeof(int64_t) * (ni + 1), st));
    query_route(q_slot, n, slot2group, gcen, it, islot2inst, q_inst, inst_qcnt, st);
    exclusive_scan_i64(inst_qcnt, q_off, ni, st, m->ar);
    CUDA_TRY(cudaMemsetAsync(inst_qcnt, 0, sizeof(int64_t) * (ni + 1), st));  // reused as cursor
    int64_t* qidx = (int64_t*)m->ar.get(Arena::kWs2, sizeof(int64_t) * std::max<int64_t>(n, 1), st);
    if (!qidx) return fail(VGP_ERR_OOM, "query index allocation failed");
    query_scatter(q_inst, n, q_off, inst_qcnt, qidx, d, grad, var, status, st);
    Q.ikeys = ikeys;
    Q.q_inst = q_inst;
    Q.inst_off = inst_off;
    Q.Xl = Xl;
    Q.Xf = Xf;
    Q.centre = centre;
    Q.gidx = gidx;
    Q.q_off = q_off;
    Q.qidx = qidx;
    return VGP_OK;
}

// Plan of a blended per-leaf G-GPDF call (Eq. 10): the node GPs (one per occupied leaf around
// the groups' centre leaves, capped to the points nearest the leaf centre) and the (query,
// node) pairs, pair id = query * n_nodes + rank, grouped by node.
struct SmoothPlan {
    GroupPlan G;
    int ni = 0;
    int64_t T = 0;
    uint64_t* ikeys = nullptr;     // node leaf key per instance
    int64_t* inst_off = nullptr;
    double* Xl = nullptr;
    float* Xf = nullptr;
    double* centre = nullptr;
    int64_t* gidx = nullptr;
    int32_t* pair_inst = nullptr;  // [n * n_nodes] node instance per (query, rank), -1 if none
    uint8_t* nn = nullptr;         // [n] nodes per query
    int64_t* q_off = nullptr;
    int64_t* qidx = nullptr;
};

static int plan_smooth(vgp_map* m, const float* q, int64_t n, int n_nodes, cudaStream_t st, SmoothPlan& SP) {
    const DevParams& P = m->P;
    GroupPlan& G = SP.G;
    TRY(plan_groups(m, q, n, st, G));
    // nodes: every occupied leaf around each group's centre leaf
    Table it;
    uint32_t Ci = pow2_at_least(2 * 27 * (int64_t)std::max(G.ng, 1));
    it.mask = Ci - 1;
    it.keys = (uint64_t*)m->ar.get(Arena::kTmp5, sizeof(uint64_t) * Ci, st);
    ARENA(islot2inst, int32_t, kTmp6, Ci);
    ARENA(ikeys, uint64_t, kTmp7, Ci);
    if (!it.keys) return fail(VGP_ERR_OOM, "node table allocation failed");
    CUDA_TRY(cudaMemsetAsync(it.keys, 0xFF, sizeof(uint64_t) * Ci, st));
    smooth_nodes(G.gcen, G.ng, m->s_tab, it, m->dev_words, st);
    collect_table(it, islot2inst, nullptr, ikeys, m->dev_words + 2, Ci, m->dev_words, st);
    TRY(read_words(m, st));
    TRY(check_err(m, "vgp_query_smooth"));
    const int ni = m->host_words[2];
    // one GP per node leaf, capped to the points nearest its centre
    ARENA(ncand, int64_t, kTmp8, ni + 1);
    ARENA(ninst, int64_t, kTmp9, ni + 1);
    ARENA(inst_off, int64_t, kTmp10, ni + 1);
    inst_count(ikeys, ni, m->s_tab, m->s_slot2leaf, m->s_off, P.cap_leaf, ncand, ninst, st, 1);
    exclusive_scan_i64(ninst, inst_off, ni, st, m->ar);
    int64_t T = 0;
    CUDA_TRY(cudaMemcpyAsync(&T, inst_off + ni, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    ARENA(Xl, double, kTmp11, 3 * T);
    ARENA(Xf, float, kTmp12, 3 * T);
    ARENA(gidx, int64_t, kTmp13, T);
    ARENA(centre, double, kTmp14, 3 * (int64_t)ni);
    inst_gather(ikeys, ni, m->s_tab, m->s_slot2leaf, m->s_off, m->s_idx, m->s_pts, ncand, inst_off, P, Xl, Xf, gidx,
                centre, st, 1);
    // (query, node) pairs grouped by node
    const int64_t np = n * n_nodes;
    ARENA(pair_inst, int32_t, kPair0, np);
    ARENA(nn, uint8_t, kPair1, n);
    ARENA(cnt, int64_t, kTmp15, ni + 1);
    ARENA(q_off, int64_t, kTmp16, ni + 1);
    ARENA(cursor, int64_t, kTmp17, ni + 1);
    ARENA(qidx, int64_t, kPair2, np);
    CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (ni + 1), st));
    CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (ni + 1), st));
    smooth_pairs(q, n, G.q_slot, G.slot2group, G.gcen, m->s_tab, it, islot2inst, P, n_nodes, pair_inst, nn, cnt, st);
    exclusive_scan_i64(cnt, q_off, ni, st, m->ar);
    smooth_scatter(pair_inst, np, q_off, cursor, qidx, st);
    SP.ni = ni;
    SP.T = T;
    SP.ikeys = ikeys;
    SP.inst_off = inst_off;
    SP.Xl = Xl;
    SP.Xf = Xf;
    SP.centre = centre;
    SP.gidx = gidx;
    SP.pair_inst = pair_inst;
    SP.nn = nn;
    SP.q_off = q_off;
    SP.qidx = qidx;
    return VGP_OK;
}

// Copy an instance table (keys, CSR offsets, global point indices) and a per-query int32 array
// to host memory (any pointer may be null), then wait for the copies.
static int copy_plan_out(const uint64_t* ikeys, const int64_t* inst_off, const int64_t* gidx, int64_t ni, int64_t T,
                         const int32_t* qa, int64_t nqa, uint64_t* key_h, int64_t* off_h, int64_t* idx_h,
                         int32_t* qa_h, cudaStream_t st) {
    if (key_h && ni) CUDA_TRY(cudaMemcpyAsync(key_h, ikeys, sizeof(uint64_t) * ni, cudaMemcpyDeviceToHost, st));
    if (off_h) CUDA_TRY(cudaMemcpyAsync(off_h, inst_off, sizeof(int64_t) * (ni + 1), cudaMemcpyDeviceToHost, st));
    if (idx_h && T) CUDA_TRY(cudaMemcpyAsync(idx_h, gidx, sizeof(int64_t) * T, cudaMemcpyDeviceToHost, st));
    if (qa_h && nqa) CUDA_TRY(cudaMemcpyAsync(qa_h, qa, sizeof(int32_t) * nqa, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return VGP_OK;
}

int vgp_query_distance_gradient(vgp_map* m, const float* q, int64_t n, double* d, double* grad, double* var,
                                uint8_t* status, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!q || !d))) return fail(VGP_ERR_ARG, "vgp_query_distance_gradient: bad argument");
    if (!m->has_surface) return fail(VGP_ERR_STATE, "vgp_query_distance_gradient before vgp_set_surface");
    if (n >= (1ll << 31)) return fail(VGP_ERR_ARG, "at most 2^31 - 1 queries per call");
    if (n == 0) return VGP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    QueryPlan Q;
    TRY(plan_queries(m, q, n, d, grad, var, status, st, Q));
    SolveBatch b;
    b.n_inst = Q.ni;
    b.inst_off = Q.inst_off;
    b.Xl = Q.Xl;
    b.Xf = Q.Xf;
    b.centre = Q.centre;
    b.q_off = Q.q_off;
    b.qidx = Q.qidx;
    b.qxyz = q;
    b.d = d;
    b.grad = grad;
    b.var = var;
    b.status = status;
    b.want_var = var != nullptr;
    SolveStats ss;
    b.max_n = m->P.cap_group;
    TRY(solve_status(solve_batch(b, m->P, m->dev_words, st, m->ar, &ss, nullptr, m->prm.profile != 0,
                                 m->prm.launch, &m->cfg, &m->gcache),
                     "query"));
    CUDA_TRY(cudaGetLastError());
    vgp_stats S{};
    S.n_points = m->s_n;
    S.n_leaves = m->s_nl;
    S.n_instances = Q.ni;
    S.n_train = Q.T;
    S.n_queries = n;
    S.n_groups = Q.ng;
    S.t_gather_ms = Q.t_gather_ms;
    S.n_candidates = Q.n_cand;
    for (int i = 0; i < 5; ++i) S.bucket_count[i] = ss.bucket_count[i];
    S.sum_n3 = ss.sum_n3;
    S.sum_n2 = ss.sum_n2;
    S.t_solve_ms = ss.t_solve_ms;
    for (int i = 0; i < 5; ++i) {
        S.t_bucket_ms[i] = ss.t_bucket_ms[i];
        S.cfg_threads[i] = m->cfg.threads[i];
        S.cfg_per_sm[i] = m->cfg.per_sm[i];
    }
    S.cfg_stage_panel = m->cfg.stage_panel;
    S.graph_replays = m->gcache.replays;
    S.graph_instantiations = m->gcache.instantiations;
    S.grid_leaves = m->g_leaves;
    S.grid_capacity_leaves = m->pool_cap;
    m->stats = S;
    return VGP_OK;
}

int vgp_query_smooth(vgp_map* m, const float* q, int64_t n, int32_t n_nodes, double lambda, double* d, double* grad,
                     double* var, uint8_t* status, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!q || !d))) return fail(VGP_ERR_ARG, "vgp_query_smooth: bad argument");
    if (n_nodes < 1 || n_nodes > 27) return fail(VGP_ERR_ARG, "vgp_query_smooth: n_nodes must be in [1, 27]");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(VGP_ERR_ARG, "vgp_query_smooth: lambda must be > 0");
    if (!m->has_surface) return fail(VGP_ERR_STATE, "vgp_query_smooth before vgp_set_surface");
    if (n == 0) return VGP_OK;
    if (n * n_nodes >= (1ll << 31)) return fail(VGP_ERR_ARG, "vgp_query_smooth: queries x nodes must be < 2^31");
    cudaStream_t st = (cudaStream_t)stream;
    const DevParams& P = m->P;
    SmoothPlan SP;
    TRY(plan_smooth(m, q, n, n_nodes, st, SP));
    const GroupPlan& G = SP.G;
    const int ni = SP.ni;
    const int64_t T = SP.T;
    const int64_t np = n * n_nodes;
    ARENA(pd, double, kPair3, np);
    ARENA(pg, double, kPair4, 3 * np);
    ARENA(ps, uint8_t, kPair5, np);
    double* pv = nullptr;
    if (var) {
        pv = (double*)m->ar.get(Arena::kPair6, sizeof(double) * np, st);
        if (!pv) return fail(VGP_ERR_OOM, "device allocation failed");
    }
    CUDA_TRY(cudaMemsetAsync(ps, 0xFF, np, st));
    SolveBatch b;
    b.n_inst = ni;
    b.inst_off = SP.inst_off;
    b.Xl = SP.Xl;
    b.Xf = SP.Xf;
    b.centre = SP.centre;
    b.q_off = SP.q_off;
    b.qidx = SP.qidx;
    b.qdiv = n_nodes;
    b.qxyz = q;
    b.d = pd;
    b.grad = pg;
    b.var = pv;
    b.status = ps;
    b.want_var = var != nullptr;
    SolveStats ss;
    b.max_n = P.cap_leaf;
    TRY(solve_status(solve_batch(b, P, m->dev_words, st, m->ar, &ss, nullptr, m->prm.profile != 0, m->prm.launch,
                                 &m->cfg, &m->gcache),
                     "vgp_query_smooth"));
    smooth_blend(n, n_nodes, G.q_slot, SP.nn, pd, pg, pv, ps, lambda, P, d, grad, var, status, st);
    CUDA_TRY(cudaGetLastError());
    vgp_stats S{};
    S.n_points = m->s_n;
    S.n_leaves = m->s_nl;
    S.n_instances = ni;
    S.n_train = T;
    S.n_queries = n;
    S.n_groups = G.ng;
    for (int i = 0; i < 5; ++i) {
        S.bucket_count[i] = ss.bucket_count[i];
        S.t_bucket_ms[i] = ss.t_bucket_ms[i];
        S.cfg_threads[i] = m->cfg.threads[i];
        S.cfg_per_sm[i] = m->cfg.per_sm[i];
    }
    S.cfg_stage_panel = m->cfg.stage_panel;
    S.graph_replays = m->gcache.replays;
    S.graph_instantiations = m->gcache.instantiations;
    S.sum_n3 = ss.sum_n3;
    S.sum_n2 = ss.sum_n2;
    S.t_solve_ms = ss.t_solve_ms;
    S.grid_leaves = m->g_leaves;
    S.grid_capacity_leaves = m->pool_cap;
    m->stats = S;
    return VGP_OK;
}

int vgp_debug_query_plan(vgp_map* m, const float* q, int64_t n, vgp_stream stream, int64_t* n_inst, int64_t* n_train,
                         uint64_t* inst_key, int64_t* inst_off, int64_t* point_idx, int32_t* q_inst) {
    if (!m || n < 0 || (n > 0 && !q) || !n_inst || !n_train) return fail(VGP_ERR_ARG, "vgp_debug_query_plan: bad argument");
    if (!m->has_surface) return fail(VGP_ERR_STATE, "vgp_debug_query_plan before vgp_set_surface");
    if (n >= (1ll << 31)) return fail(VGP_ERR_ARG, "at most 2^31 - 1 queries per call");
    *n_inst = 0;
    *n_train = 0;
    if (n == 0) return VGP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    double* dtmp = (double*)m->ar.get(Arena::kBw0, sizeof(double) * n, st);
    if (!dtmp) return fail(VGP_ERR_OOM, "allocation failed");
    QueryPlan Q;
    TRY(plan_queries(m, q, n, dtmp, nullptr, nullptr, nullptr, st, Q));
    *n_inst = Q.ni;
    *n_train = Q.T;
    return copy_plan_out(Q.ikeys, Q.inst_off, Q.gidx, Q.ni, Q.T, Q.q_inst, n, inst_key, inst_off, point_idx, q_inst, st);
}

int vgp_debug_smooth_plan(vgp_map* m, const float* q, int64_t n, int32_t n_nodes, vgp_stream stream, int64_t* n_inst,
                          int64_t* n_train, uint64_t* node_key, int64_t* inst_off, int64_t* point_idx,
                          int32_t* pair_inst) {
    if (!m || n < 0 || (n > 0 && !q) || !n_inst || !n_train) return fail(VGP_ERR_ARG, "vgp_debug_smooth_plan: bad argument");
    if (n_nodes < 1 || n_nodes > 27) return fail(VGP_ERR_ARG, "vgp_debug_smooth_plan: n_nodes must be in [1, 27]");
    if (!m->has_surface) return fail(VGP_ERR_STATE, "vgp_debug_smooth_plan before vgp_set_surface");
    if (n * n_nodes >= (1ll << 31)) return fail(VGP_ERR_ARG, "vgp_debug_smooth_plan: queries x nodes must be < 2^31");
    *n_inst = 0;
    *n_train = 0;
    if (n == 0) return VGP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    SmoothPlan SP;
    TRY(plan_smooth(m, q, n, n_nodes, st, SP));
    *n_inst = SP.ni;
    *n_train = SP.T;
    return copy_plan_out(SP.ikeys, SP.inst_off, SP.gidx, SP.ni, SP.T, SP.pair_inst, n * n_nodes, node_key, inst_off,
                         point_idx, pair_inst, st);
}

int vgp_autotune(vgp_map* m, const float* q, int64_t n, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && !q)) return fail(VGP_ERR_ARG, "vgp_autotune: bad argument");
    if (!m->has_surface) return fail(VGP_ERR_STATE, "vgp_autotune before vgp_set_surface");
    if (n == 0) return VGP_OK;
    if (n >= (1ll << 31)) return fail(VGP_ERR_ARG, "at most 2^31 - 1 queries per call");
    cudaStream_t st = (cudaStream_t)stream;
    double* dtmp = (double*)m->ar.get(Arena::kBw0, sizeof(double) * n, st);
    if (!dtmp) return fail(VGP_ERR_OOM, "allocation failed");
    QueryPlan Q;
    TRY(plan_queries(m, q, n, dtmp, nullptr, nullptr, nullptr, st, Q));
    SolveBatch b;
    b.n_inst = Q.ni;
    b.inst_off = Q.inst_off;
    b.Xl = Q.Xl;
    b.Xf = Q.Xf;
    b.centre = Q.centre;
    b.q_off = Q.q_off;
    b.qidx = Q.qidx;
    b.qxyz = q;
    b.d = dtmp;
    // candidate launch shapes (threads per CTA, CTAs per SM cap) per size bucket
    // (the last three: N > 224 without panel staging, two or three CTAs per SM)
    const int cand_t[7][5] = {{512, 512, 256, 128, 64}, {256, 256, 128, 64, 32}, {256, 384, 512, 256, 128},
                              {128, 128, 64, 32, 256},  {384, 512, 256, 128, 64}, {256, 512, 256, 128, 64},
                              {256, 512, 256, 128, 64}};
    const int cand_p[7][5] = {{1, 0, 0, 0, 0}, {2, 0, 0, 0, 0}, {1, 0, 0, 0, 0}, {4, 0, 0, 0, 0},
                              {2, 0, 0, 0, 0}, {2, 0, 0, 0, 0}, {3, 0, 0, 0, 0}};
    const int cand_s[7] = {1, 1, 1, 1, 0, 0, 0};
    double best[5] = {1e300, 1e300, 1e300, 1e300, 1e300};
    SolveConfig chosen = m->cfg;
    for (int c = 0; c < 7; ++c) {
        SolveConfig cfg;
        for (int i = 0; i < 5; ++i) {
            cfg.threads[i] = cand_t[c][i];
            cfg.per_sm[i] = cand_p[c][i];
        }
        cfg.stage_panel = cand_s[c];
        // each candidate twice, the faster run counts
        SolveStats s1, s2;
        TRY(solve_status(solve_batch(b, m->P, m->dev_words, st, m->ar, &s1, nullptr, true, 0, &cfg), "vgp_autotune"));
        TRY(solve_status(solve_batch(b, m->P, m->dev_words, st, m->ar, &s2, nullptr, true, 0, &cfg), "vgp_autotune"));
        CUDA_TRY(cudaGetLastError());
        SolveStats ss = s1;
        for (int i = 0; i < 5; ++i) ss.t_bucket_ms[i] = std::min(s1.t_bucket_ms[i], s2.t_bucket_ms[i]);
        for (int i = 0; i < 5; ++i)
            if (ss.bucket_count[i] > 0 && ss.t_bucket_ms[i] < best[i]) {
                best[i] = ss.t_bucket_ms[i];
                chosen.threads[i] = cfg.threads[i];
                chosen.per_sm[i] = cfg.per_sm[i];
                if (i == 0) chosen.stage_panel = cfg.stage_panel;
            }
    }
    m->cfg = chosen;
    for (int i = 0; i < 5; ++i) {
        m->stats.cfg_threads[i] = chosen.threads[i];
        m->stats.cfg_per_sm[i] = chosen.per_sm[i];
        m->stats.t_bucket_ms[i] = best[i] < 1e299 ? best[i] : 0.0;
    }
    m->stats.cfg_stage_panel = chosen.stage_panel;
    return VGP_OK;
}

int vgp_set_launch(vgp_map* m, const int32_t* threads, const int32_t* per_sm, int32_t stage_panel) {
    if (!m || !threads || !per_sm || (stage_panel != 0 && stage_panel != 1))
        return fail(VGP_ERR_ARG, "vgp_set_launch: bad argument");
    for (int i = 0; i < 5; ++i) {
        if (threads[i] < 32 || threads[i] > 1024 || threads[i] % 32 != 0)
            return fail(VGP_ERR_ARG, "vgp_set_launch: threads must be multiples of 32 in [32, 1024]");
        if (per_sm[i] < 0 || per_sm[i] > 32) return fail(VGP_ERR_ARG, "vgp_set_launch: per_sm must be in [0, 32]");
    }
    for (int i = 0; i < 5; ++i) {
        m->cfg.threads[i] = threads[i];
        m->cfg.per_sm[i] = per_sm[i];
    }
    m->cfg.stage_panel = stage_panel;
    return VGP_OK;
}

int vgp_query_backward(vgp_map* m, const float* q, int64_t n, const double* dL_dd, double* dL_dq, double* dL_dX,
                       vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!q || !dL_dd))) return fail(VGP_ERR_ARG, "vgp_query_backward: bad argument");
    if (!m->has_surface) return fail(VGP_ERR_STATE, "vgp_query_backward before vgp_set_surface");
    if (n >= (1ll << 31)) return fail(VGP_ERR_ARG, "at most 2^31 - 1 queries per call");
    cudaStream_t st = (cudaStream_t)stream;
    if (dL_dq && n > 0) CUDA_TRY(cudaMemsetAsync(dL_dq, 0, sizeof(double) * 3 * n, st));
    if (dL_dX && m->s_n > 0) CUDA_TRY(cudaMemsetAsync(dL_dX, 0, sizeof(double) * 3 * m->s_n, st));
    if (n == 0) return VGP_OK;
    double* dtmp = (double*)m->ar.get(Arena::kBw0, sizeof(double) * n, st);
    if (!dtmp) return fail(VGP_ERR_OOM, "allocation failed");
    QueryPlan Q;
    TRY(plan_queries(m, q, n, dtmp, nullptr, nullptr, nullptr, st, Q));
    double* obar = (double*)m->ar.get(Arena::kBw1, sizeof(double) * n, st);
    if (!obar) return fail(VGP_ERR_OOM, "allocation failed");
    SolveBatch b;
    b.n_inst = Q.ni;
    b.inst_off = Q.inst_off;
    b.Xl = Q.Xl;
    b.Xf = Q.Xf;
    b.centre = Q.centre;
    b.q_off = Q.q_off;
    b.qidx = Q.qidx;
    b.qxyz = q;
    b.d = dtmp;
    BackwardBatch bw;
    bw.gidx = Q.gidx;
    bw.dL_dd = dL_dd;
    bw.dL_dq = dL_dq;
    bw.dL_dX = dL_dX;
    bw.obar = obar;
    TRY(solve_status(solve_batch(b, m->P, m->dev_words, st, m->ar, nullptr, &bw, false, 0, &m->cfg),
                     "vgp_query_backward"));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaGetLastError());
    return VGP_OK;
}

}  // extern "C"

// ---------------------------------- independent instances ------------------------------
namespace {
// Warp per instance: bounds check, bounding-box centre, local coordinates.
__global__ void k_batch_prep(const int64_t* inst_off, int64_t n_inst, const float* X, double* Xl, float* Xf,
                             double* centre, int* err) {
    int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (I >= n_inst) return;
    const int64_t b = inst_off[I], e = inst_off[I + 1];
    if (e - b > 1024 || e < b) {
        if (lane == 0) atomicOr(err, kErrCapacity);
        return;
    }
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = b + lane; j < e; j += 32)
        for (int a = 0; a < 3; ++a) {
            float v = X[3 * j + a];
            lo[a] = fminf(lo[a], v);
            hi[a] = fmaxf(hi[a], v);
        }
    double c[3];
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        c[a] = (e > b && isfinite(lo[a]) && isfinite(hi[a])) ? 0.5 * ((double)lo[a] + (double)hi[a]) : 0.0;
    }
    if (lane < 3) centre[3 * I + lane] = c[lane];
    for (int64_t j = b + lane; j < e; j += 32)
        for (int a = 0; a < 3; ++a) {
            double v = (double)X[3 * j + a] - c[a];
            Xl[3 * j + a] = v;
            Xf[3 * j + a] = (float)v;
        }
}
}  // namespace

namespace {
__global__ void k_exp_probe(const double* y, double* out, int64_t n, const double* tab) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = exp_neg(y[i], tab);
}
}  // namespace

extern "C" int vgp_debug_exp_neg(const vgp_map* m, const double* y, double* out, int64_t n, vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!y || !out))) return fail(VGP_ERR_ARG, "vgp_debug_exp_neg: bad argument");
    if (n == 0) return VGP_OK;
    k_exp_probe<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(y, out, n, m->P.exp_tab);
    note_launch();
    CUDA_TRY(cudaGetLastError());
    return VGP_OK;
}

extern "C" int vgp_debug_kernel_fix(const vgp_map* m, const float* xa, const float* xb, int64_t n, int64_t* out,
                                    vgp_stream stream) {
    if (!m || n < 0 || (n > 0 && (!xa || !xb || !out))) return fail(VGP_ERR_ARG, "vgp_debug_kernel_fix: bad argument");
    if (debug_kernel_fix(m->P, xa, xb, n, (long long*)out, (cudaStream_t)stream) != 0)
        return fail(VGP_ERR_CUDA, "vgp_debug_kernel_fix: launch failed");
    return VGP_OK;
}

extern "C" int vgp_gp_batch(vgp_map* m, int64_t n_inst, const int64_t* inst_off, const float* X, const int64_t* q_off,
                            const float* Q, double* d, double* grad, double* var, uint8_t* status, vgp_stream stream) {
    if (!m || n_inst < 0 || (n_inst > 0 && (!inst_off || !q_off || !d)))
        return fail(VGP_ERR_ARG, "vgp_gp_batch: bad argument");
    if (n_inst == 0) return VGP_OK;
    if (n_inst >= (1ll << 31)) return fail(VGP_ERR_ARG, "vgp_gp_batch: too many instances");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t T = 0, NQ = 0;
    CUDA_TRY(cudaMemcpyAsync(&T, inst_off + n_inst, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&NQ, q_off + n_inst, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (T < 0 || NQ < 0) return fail(VGP_ERR_ARG, "vgp_gp_batch: negative totals");
    CUDA_TRY(cudaMemsetAsync(m->dev_words, 0, sizeof(int) * 8, st));
    ARENA(Xl, double, kTmp11, 3 * T);
    ARENA(Xf, float, kTmp12, 3 * T);
    ARENA(centre, double, kTmp14, 3 * n_inst);
    k_batch_prep<<<(unsigned)((n_inst * 32 + 255) / 256), 256, 0, st>>>(inst_off, n_inst, X, Xl, Xf, centre,
                                                                         m->dev_words);
    note_launch();
    TRY(read_words(m, st));
    if (m->host_words[0] & kErrCapacity) return fail(VGP_ERR_ARG, "vgp_gp_batch: an instance has more than 1024 points");
    SolveBatch b;
    b.n_inst = n_inst;
    b.inst_off = inst_off;
    b.Xl = Xl;
    b.Xf = Xf;
    b.centre = centre;
    b.q_off = q_off;
    b.qidx = nullptr;
    b.qxyz = Q;
    b.d = d;
    b.grad = grad;
    b.var = var;
    b.status = status;
    b.want_var = var != nullptr;
    SolveStats ss;
    TRY(solve_status(solve_batch(b, m->P, m->dev_words, st, m->ar, &ss, nullptr, m->prm.profile != 0,
                                 m->prm.launch, &m->cfg, &m->gcache),
                     "vgp_gp_batch"));
    CUDA_TRY(cudaGetLastError());
    vgp_stats S{};
    S.n_instances = n_inst;
    S.n_train = T;
    S.n_queries = NQ;
    for (int i = 0; i < 5; ++i) S.bucket_count[i] = ss.bucket_count[i];
    S.sum_n3 = ss.sum_n3;
    S.sum_n2 = ss.sum_n2;
    S.t_solve_ms = ss.t_solve_ms;
    for (int i = 0; i < 5; ++i) {
        S.t_bucket_ms[i] = ss.t_bucket_ms[i];
        S.cfg_threads[i] = m->cfg.threads[i];
        S.cfg_per_sm[i] = m->cfg.per_sm[i];
    }
    S.cfg_stage_panel = m->cfg.stage_panel;
    S.graph_replays = m->gcache.replays;
    S.graph_instantiations = m->gcache.instantiations;
    m->stats = S;
    return VGP_OK;
}
