// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"

namespace vgp {

// Stream-ordered scratch buffers that grow on demand (cudaMallocAsync on the call's stream).
class Arena {
public:
    enum Slot {
        kScan0, kScan1, kScan2, kHist, kOrder, kTmp0, kTmp1, kTmp2, kTmp3, kTmp4, kTmp5, kTmp6,
        kTmp7, kTmp8, kTmp9, kTmp10, kTmp11, kTmp12, kTmp13, kTmp14, kTmp15, kTmp16, kTmp17,
        kWs0, kWs1, kWs2, kWs3, kBw0, kBw1, kPair0, kPair1, kPair2, kPair3, kPair4, kPair5, kPair6, kPair7,
        kChunks, kCounters, kNumSlots
    };
    void* get(Slot s, size_t bytes, cudaStream_t st);
    void release_all(cudaStream_t st);
    ~Arena();

private:
    void* ptr_[kNumSlots] = {};
    size_t size_[kNumSlots] = {};
};

// Instances to solve (one GP each) with the queries that each must answer.
struct SolveBatch {
    int64_t n_inst = 0;
    const int64_t* inst_off = nullptr;  // [n_inst + 1] offsets into Xl / Xf
    const double* Xl = nullptr;         // [T][3] FP64 coordinates relative to the centre
    const float* Xf = nullptr;          // [T][3] FP32 copy of Xl
    const double* centre = nullptr;     // [n_inst][3] FP64 world-frame centre
    const char4* Xi = nullptr;          // lattice instances: in-leaf voxel offsets (0..7) per point
    const uint64_t* inst_key = nullptr; // lattice instances: leaf key of each instance
    const int64_t* q_off = nullptr;     // [n_inst + 1] offsets into the position list
    const int64_t* qidx = nullptr;      // position -> query id (nullptr: identity)
    int qdiv = 1;                       // query point of id q is qxyz[q / qdiv] (pairs)
    const float* qxyz = nullptr;        // world-frame query points (by query id)
    const uint64_t* qkey = nullptr;     // voxel-key queries (by position), if qxyz is null
    double* d = nullptr;                // outputs by query id
    double* grad = nullptr;
    double* var = nullptr;
    uint8_t* status = nullptr;
    double* alpha_out = nullptr;        // [T] optional
    int want_var = 0;
    // surface-property mode (Eq. 6): nprop > 0 replaces the right-hand side 1 by the nprop
    // columns of yprop and writes property means / variances instead of distances
    int nprop = 0;
    int max_n = 1024;                   // largest N the batch can hold (sizes graph-mode buffers)
    const double* yprop = nullptr;      // [T][nprop]
    double* pc = nullptr;               // [n_queries][nprop] by query id
    double* pw = nullptr;               // [n_queries] by query id
};

// Backward-pass extras (G-GPDF only).
struct BackwardBatch {
    const int64_t* gidx = nullptr;  // [T] global surface index of each instance point
    const double* dL_dd = nullptr;  // [n_queries] by query id
    double* dL_dq = nullptr;        // [n_queries][3]
    double* dL_dX = nullptr;        // [n_surface][3] accumulated with atomics
    double* obar = nullptr;         // [n_positions] scratch
};

// Launch shape of the five size buckets of solve_batch (N > 224 with A in global memory,
// then N <= 224, 128, 64, 32 with A in shared memory): threads per CTA and the cap on
// resident CTAs per SM (0: as many as fit).  Chosen by vgp_autotune or the defaults.  With
// emulate_fp64 the buckets above 32 points run the emulated kernel, whose shape is fixed.
struct SolveConfig {
    int threads[5] = {512, 512, 256, 128, 64};
    int per_sm[5] = {1, 0, 0, 0, 0};
    // N > 224 (A in global memory): stage the current panel column in shared memory (1), or
    // read it from the global tile-packed matrix through L1/L2 (0), which leaves room for two
    // CTAs per SM
    int stage_panel = 1;
};

struct SolveStats {
    int64_t bucket_count[5] = {0, 0, 0, 0, 0};
    double t_bucket_ms[5] = {0, 0, 0, 0, 0};  // per bucket, when profiling
    double sum_n3 = 0;
    double sum_n2 = 0;
    double t_solve_ms = 0;  // filled when profiling
};

// Process-wide count of kernel launches (each launch site calls this once).
void note_launch();

// scan.cu / grid kernels
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st, Arena& ar);
void fill_i64(int64_t* p, int64_t v, int64_t n, cudaStream_t st);
void fill_u64(uint64_t* p, uint64_t v, int64_t n, cudaStream_t st);
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t st);
void widen_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t st);

// CUDA-graph state of a map (launch mode VGP_LAUNCH_GRAPH): a private capture stream, two
// events joining it to the caller's stream, and one executable graph per solve kind.
struct GraphCache {
    cudaStream_t gs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};  // distance, surface property
    int64_t replays = 0, instantiations = 0;
};
void graph_cache_destroy(GraphCache& gc);

// Solve every instance of the batch (factorise, alpha, evaluate its queries).  Returns
// error bits through *err_dev.  Synchronises once to read the size histogram (in graph mode
// the histogram is planned on the device and read once at the end, for the statistics).
// Returns 0; -1 when graph capture, instantiation or launch failed (kErrLaunch is then also
// set in *err_dev); -2 when a workspace could not be allocated (kErrAlloc is set in *err_dev
// and no solve kernel was launched).
int solve_batch(const SolveBatch& b, const DevParams& P, int* err_dev, cudaStream_t st,
                 Arena& ar, SolveStats* stats, const BackwardBatch* bw = nullptr, bool profile = false,
                 int launch = 0, const SolveConfig* cfg = nullptr, GraphCache* gc = nullptr);

// Set the thread-local message returned by vgp_last_error().
void set_last_error(const char* msg);

// Diagnostic: the emulated kernel's mixed-precision kernel values round(k 2^61) of n pairs of
// FP32 world coordinates (device arrays [n][3]); 0 or -1 on a launch error.
int debug_kernel_fix(const DevParams& P, const float* xa, const float* xb, int64_t n, long long* out,
                     cudaStream_t st);

// k_solve with caller-provided scratch and no allocation (see noalloc.cu); 0 on success.
int solve_launch_static(const SolveBatch& b, const DevParams& P, int* err_dev, int npad, int threads, int max_grid,
                        int* counter, const int32_t* order, double* ws_v, cudaStream_t st);

}  // namespace vgp
