// noalloc.cu -- vgp_gp_batch_static: the batched GP solve for callers that cannot allocate
// device memory (code running inside a captured or externally managed memory regime, an
// embedded host with a fixed memory budget, or a caller that must never trigger cudaMalloc).
//
// All scratch lives in one file-scope __device__ array of kScratchBytes.  The array's name
// is only a host-side stand-in for it in host code, so host code asks the runtime for its
// device address (cudaGetSymbolAddress) once per device, with that device current, and
// passes that address to the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace {

using namespace vgp;

constexpr int64_t kMaxInst = 1 << 16;    // instances per call
constexpr int64_t kMaxPoints = 1 << 18;  // training points per call (sum of N)
constexpr int kMaxN = 64;                // points per instance
constexpr int kThreads = 128;            // threads per CTA
constexpr int kMaxGrid = 304;            // persistent CTAs (2 per SM on 152 SMs)

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffWords = 0;                                                  // [0] counter, [1] error
constexpr size_t kOffTab = 256;                                                  // 2^(j/256), 256 doubles
constexpr size_t kOffOrder = align256(kOffTab + 256 * sizeof(double));           // int32 per instance
constexpr size_t kOffCentre = align256(kOffOrder + kMaxInst * sizeof(int32_t));  // 3 doubles per instance
constexpr size_t kOffXl = align256(kOffCentre + 3 * kMaxInst * sizeof(double));  // 3 doubles per point
constexpr size_t kOffXf = align256(kOffXl + 3 * kMaxPoints * sizeof(double));    // 3 floats per point
constexpr size_t kOffV = align256(kOffXf + 3 * kMaxPoints * sizeof(float));      // variance columns
constexpr size_t kScratchBytes = kOffV + (size_t)kMaxGrid * kMaxN * kThreads * sizeof(double);  // ~30.7 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
unsigned char* g_ptr[256] = {};  // device address of g_scratch per device ordinal

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

// 2^(j/256), j = 0..255, for the FP64 table exponential; written into the scratch array on the
// caller's stream by every call (stream-ordered, so no stream can read it half written).
struct ExpTable {
    double v[256];
    ExpTable() {
        for (int j = 0; j < 256; ++j) v[j] = (double)exp2l((long double)j / 256.0L);
    }
};
const ExpTable g_tab;

// Device address of the scratch array on the current device, looked up once per device (the
// first call on that device) with that device current.
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(VGP_ERR_CUDA, "vgp_gp_batch_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(VGP_ERR_ARG, "vgp_gp_batch_static: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(VGP_ERR_CUDA, "vgp_gp_batch_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_ptr[dev] = (unsigned char*)p;
    }
    *out = g_ptr[dev];
    return VGP_OK;
}

// error bits of k_static_prep
constexpr int kBadOffsets = 1;  // inst_off[I] < 0, inst_off[I+1] < inst_off[I], or beyond kMaxPoints
constexpr int kTooLarge = 2;    // an instance with more than kMaxN points

// Warp per instance: offset and size checks, bounding-box centre, local coordinates, identity
// order.  A rejected instance writes nothing into the scratch array.
__global__ void k_static_prep(const int64_t* inst_off, int64_t n_inst, const float* X, double* Xl, float* Xf,
                              double* centre, int32_t* order, int* err) {
    const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (I >= n_inst) return;
    const int64_t b = inst_off[I], e = inst_off[I + 1];
    if (lane == 0) order[I] = (int32_t)I;
    if (b < 0 || e < b || e > kMaxPoints) {
        if (lane == 0) atomicOr(err, kBadOffsets);
        return;
    }
    if (e - b > kMaxN) {
        if (lane == 0) atomicOr(err, kTooLarge);
        return;
    }
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = b + lane; j < e; j += 32)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], X[3 * j + a]);
            hi[a] = fmaxf(hi[a], X[3 * j + a]);
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
            const double v = (double)X[3 * j + a] - c[a];
            Xl[3 * j + a] = v;
            Xf[3 * j + a] = (float)v;
        }
}

bool params_ok(const vgp_params* p) {
    return p && p->voxel_size > 0 && std::isfinite(p->voxel_size) && p->lengthscale > 0 && std::isfinite(p->lengthscale) &&
           p->sigma_occ > 0 && std::isfinite(p->sigma_occ) && p->d_max > 0 && p->d_var_floor > 0 &&
           (p->precision == VGP_FP64 || p->precision == VGP_MIXED);
}

}  // namespace

extern "C" int vgp_gp_batch_static(const vgp_params* p, int64_t n_inst, const int64_t* inst_off, const float* X,
                                   const int64_t* q_off, const float* Q, double* d, double* grad, double* var,
                                   uint8_t* status, vgp_stream stream) {
    if (!params_ok(p)) return fail(VGP_ERR_ARG, "vgp_gp_batch_static: invalid parameters");
    if (n_inst < 0 || (n_inst > 0 && (!inst_off || !q_off || !X || !Q || !d)))
        return fail(VGP_ERR_ARG, "vgp_gp_batch_static: bad argument");
    if (n_inst > kMaxInst)
        return fail(VGP_ERR_ARG, "vgp_gp_batch_static: %lld instances exceed the maximum of %lld", (long long)n_inst,
                    (long long)kMaxInst);
    if (n_inst == 0) return VGP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != VGP_OK) return rc;
    int64_t T = 0;
    cudaError_t e = cudaMemcpyAsync(&T, inst_off + n_inst, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(VGP_ERR_CUDA, "vgp_gp_batch_static: %s", cudaGetErrorString(e));
    if (T < 0 || T > kMaxPoints)
        return fail(VGP_ERR_ARG, "vgp_gp_batch_static: %lld training points exceed the maximum of %lld", (long long)T,
                    (long long)kMaxPoints);
    int* words = (int*)(base + kOffWords);
    double* Xl = (double*)(base + kOffXl);
    float* Xf = (float*)(base + kOffXf);
    double* centre = (double*)(base + kOffCentre);
    int32_t* order = (int32_t*)(base + kOffOrder);
    double* V = (double*)(base + kOffV);
    e = cudaMemsetAsync(words, 0, 2 * sizeof(int), st);  // work counter and error word start at zero
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffTab, g_tab.v, sizeof(g_tab.v), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(VGP_ERR_CUDA, "vgp_gp_batch_static: %s", cudaGetErrorString(e));
    k_static_prep<<<(unsigned)((n_inst * 32 + 255) / 256), 256, 0, st>>>(inst_off, n_inst, X, Xl, Xf, centre, order,
                                                                          words + 1);
    note_launch();
    int h_err = 0;
    e = cudaMemcpyAsync(&h_err, words + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(VGP_ERR_CUDA, "vgp_gp_batch_static: %s", cudaGetErrorString(e));
    if (h_err & kBadOffsets)
        return fail(VGP_ERR_ARG, "vgp_gp_batch_static: inst_off is negative, decreasing or beyond %lld points",
                    (long long)kMaxPoints);
    if (h_err) return fail(VGP_ERR_ARG, "vgp_gp_batch_static: an instance has more than %d points", kMaxN);
    DevParams P{};
    P.vs = p->voxel_size;
    P.l = p->lengthscale;
    P.l2 = p->lengthscale * p->lengthscale;
    P.inv2l2 = 1.0 / (2.0 * P.l2);
    P.s2 = p->sigma_occ * p->sigma_occ;
    P.d_max = p->d_max;
    P.log_floor = -(p->d_max * p->d_max) / (2.0 * P.l2);
    P.d_var_floor = p->d_var_floor;
    P.inv2l2_log2e = (float)(1.4426950408889634 / (2.0 * P.l2));
    P.inv2l2_hi = (float)P.inv2l2;
    P.inv2l2_lo = (float)(P.inv2l2 - (double)P.inv2l2_hi);
    P.vs_f = (float)p->voxel_size;
    P.precision = p->precision;
    P.exp_tab = (const double*)(base + kOffTab);
    SolveBatch b;
    b.n_inst = n_inst;
    b.inst_off = inst_off;
    b.Xl = Xl;
    b.Xf = Xf;
    b.centre = centre;
    b.q_off = q_off;
    b.qxyz = Q;
    b.d = d;
    b.grad = grad;
    b.var = var;
    b.status = status;
    b.want_var = var != nullptr;
    if (solve_launch_static(b, P, words + 1, kMaxN, kThreads, kMaxGrid, words, order, V, st) != 0)
        return fail(VGP_ERR_CUDA, "vgp_gp_batch_static: launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return VGP_OK;
}
