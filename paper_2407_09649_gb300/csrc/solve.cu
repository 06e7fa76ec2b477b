// solve.cu -- batched GP instances: K assembly, FP64 Cholesky, alpha, and the fused
// evaluation of every query of the instance (latent mean Eq. 1, variance Eq. 2, gradient
// Eq. 5, reverting Eq. 3 and distance variance Eq. 4), plus the backward pass.
//
// One CTA owns one instance at a time and pulls instances from a list sorted by
// decreasing size (a persistent launch per size bucket, longest-first).  The packed lower
// triangle of A = K + sigma^2 I lives in shared memory when it fits, else in a per-CTA
// global workspace.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "internal.h"

namespace vgp {

namespace {

__host__ __device__ __forceinline__ int64_t pk(int i, int j) { return (int64_t)i * (i + 1) / 2 + j; }

struct SolveCtx {
    SolveBatch b;
    DevParams P;
    int* err;
    int* counter;
    const int32_t* order;  // instance ids, decreasing N
    int n_work;
    int nmax;              // largest N in this launch
    int a_in_smem;
    double* ws_a;          // per-CTA packed A when not in shared memory
    int64_t ws_a_stride;
    double* ws_v;          // per-CTA variance columns [nmax][blockDim]
    int64_t ws_v_stride;
    BackwardBatch bw;
    int backward;
};

struct Shared {
    double* X;      // [N][3] local FP64
    double* alpha;  // [N]
    double* invd;   // [N] 1 / L_ii
    double* y;      // [N] scratch
    double* z;      // [N] scratch
    double* A;      // packed lower triangle
    float* Xf;      // [N][3]
    float* alf;     // [N]
};

__device__ Shared carve(double* sm, int nmax, int a_in_smem, double* ws_a) {
    Shared s;
    s.X = sm;
    s.alpha = s.X + 3 * nmax;
    s.invd = s.alpha + nmax;
    s.y = s.invd + nmax;
    s.z = s.y + nmax;
    double* end = s.z + nmax;
    if (a_in_smem) {
        s.A = end;
        end += pk(nmax, 0);
    } else {
        s.A = ws_a;
    }
    s.Xf = reinterpret_cast<float*>(end);
    s.alf = s.Xf + 3 * nmax;
    return s;
}

__host__ size_t smem_bytes(int nmax, int a_in_smem) {
    size_t d = (size_t)7 * nmax + (a_in_smem ? (size_t)pk(nmax, 0) : 0);
    return d * sizeof(double) + (size_t)4 * nmax * sizeof(float);
}

// Assemble A, factorise, solve alpha.  Returns false if a pivot was not positive.
__device__ bool fit_instance(const SolveCtx& c, const Shared& s, int I, int N, int64_t base) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_fail;
    for (int t = tid; t < 3 * N; t += nt) {
        double v = c.b.Xl[3 * base + t];
        s.X[t] = v;
        s.Xf[t] = (float)v;
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    double* A = s.A;
    // K + sigma^2 I, lower triangle (Sec. III-A kernel, Eq. 1 noise term)
    const int TX = 16, TY = nt / 16;
    const int tx = tid % TX, ty = tid / TX;
    for (int i = ty; i < N; i += TY) {
        const double xi = s.X[3 * i], yi = s.X[3 * i + 1], zi = s.X[3 * i + 2];
        for (int j = tx; j <= i; j += TX) {
            double v;
            if (j == i) {
                v = 1.0 + c.P.s2;
            } else {
                double dx = xi - s.X[3 * j], dy = yi - s.X[3 * j + 1], dz = zi - s.X[3 * j + 2];
                double r2 = dx * dx + dy * dy + dz * dz;
                v = exp(-r2 * c.P.inv2l2);
            }
            A[pk(i, j)] = v;
        }
    }
    __syncthreads();
    // right-looking Cholesky, column by column
    for (int k = 0; k < N; ++k) {
        if (tid == 0) {
            double a = A[pk(k, k)];
            if (!(a > 0.0)) {
                s_fail = 1;
            } else {
                double r = sqrt(a);
                A[pk(k, k)] = r;
                s.invd[k] = 1.0 / r;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double ik = s.invd[k];
        for (int i = k + 1 + tid; i < N; i += nt) A[pk(i, k)] *= ik;
        __syncthreads();
        for (int i = k + 1 + ty; i < N; i += TY) {
            const double lik = A[pk(i, k)];
            for (int j = k + 1 + tx; j <= i; j += TX) A[pk(i, j)] -= lik * A[pk(j, k)];
        }
        __syncthreads();
    }
    if (s_fail) return false;
    // alpha = L^-T L^-1 1 (Eq. 1)
    for (int i = tid; i < N; i += nt) s.z[i] = 1.0;
    __syncthreads();
    for (int j = 0; j < N; ++j) {
        const double yj = s.z[j] * s.invd[j];
        for (int i = j + 1 + tid; i < N; i += nt) s.z[i] -= A[pk(i, j)] * yj;
        if (tid == 0) s.y[j] = yj;
        __syncthreads();
    }
    for (int j = N - 1; j >= 0; --j) {
        const double aj = s.y[j] * s.invd[j];
        for (int i = tid; i < j; i += nt) s.y[i] -= A[pk(j, i)] * aj;
        __syncthreads();
        if (tid == 0) s.alpha[j] = aj;
        __syncthreads();
    }
    for (int j = tid; j < N; j += nt) s.alf[j] = (float)s.alpha[j];
    __syncthreads();
    return true;
}

struct EvalOut {
    double d, g[3], v;
    int status;
};

// Reverting (Eq. 3), distance variance (Eq. 4), chain-rule gradient, with the caps of the
// occupancy: lo = log o, gro = grad o / o.
__device__ __forceinline__ void revert(const DevParams& P, double lo, const double gro[3], double u,
                                       bool want_var, EvalOut& r) {
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

__device__ __forceinline__ void query_local(const SolveCtx& c, int I, int64_t p, int64_t qid, double xl[3]) {
    double xg[3];
    if (c.b.qkey) {
        int i, j, k;
        unpack_key(c.b.qkey[p], i, j, k);
        xg[0] = (double)i * c.P.vs;
        xg[1] = (double)j * c.P.vs;
        xg[2] = (double)k * c.P.vs;
    } else {
        xg[0] = (double)c.b.qxyz[3 * qid];
        xg[1] = (double)c.b.qxyz[3 * qid + 1];
        xg[2] = (double)c.b.qxyz[3 * qid + 2];
    }
    for (int a = 0; a < 3; ++a) xl[a] = xg[a] - c.b.centre[3 * (int64_t)I + a];
}

// Latent mean and gradient at one query; returns lo = log o and gro = grad o / o.
__device__ __forceinline__ void latent_mean(const SolveCtx& c, const Shared& s, int N, const double xl[3],
                                            double& lo, double gro[3]) {
    if (c.P.precision == VGP_MIXED) {
        // FP32 with the nearest training point as the shift: exp(-(r^2 - r0^2) / 2l^2) <= 1
        const float qx = (float)xl[0], qy = (float)xl[1], qz = (float)xl[2];
        float r0 = INFINITY;
        for (int j = 0; j < N; ++j) {
            float dx = s.Xf[3 * j] - qx, dy = s.Xf[3 * j + 1] - qy, dz = s.Xf[3 * j + 2] - qz;
            r0 = fminf(r0, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
        float sum = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        for (int j = 0; j < N; ++j) {
            float dx = s.Xf[3 * j] - qx, dy = s.Xf[3 * j + 1] - qy, dz = s.Xf[3 * j + 2] - qz;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float w = s.alf[j] * exp2f((r0 - r2) * c.P.inv2l2_log2e);
            sum += w;
            gx = fmaf(w, dx, gx);
            gy = fmaf(w, dy, gy);
            gz = fmaf(w, dz, gz);
        }
        if (!(sum > 0.f)) {
            lo = NAN;
            gro[0] = gro[1] = gro[2] = 0.0;
            return;
        }
        lo = -(double)r0 * c.P.inv2l2 + log((double)sum);
        const double inv = 1.0 / ((double)sum * c.P.l2);
        gro[0] = (double)gx * inv;
        gro[1] = (double)gy * inv;
        gro[2] = (double)gz * inv;
    } else {
        double o = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int j = 0; j < N; ++j) {
            double dx = s.X[3 * j] - xl[0], dy = s.X[3 * j + 1] - xl[1], dz = s.X[3 * j + 2] - xl[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double w = s.alpha[j] * exp(-r2 * c.P.inv2l2);
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
        const double inv = 1.0 / (o * c.P.l2);
        gro[0] = gx * inv;
        gro[1] = gy * inv;
        gro[2] = gz * inv;
    }
}

// u = 1 - |L^-1 k|^2 (Eq. 2), the thread's own column of V in global workspace.
__device__ __forceinline__ double latent_var(const SolveCtx& c, const Shared& s, int N, const double xl[3],
                                             double* V, int stride) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
        double dx = s.X[3 * i] - xl[0], dy = s.X[3 * i + 1] - xl[1], dz = s.X[3 * i + 2] - xl[2];
        double sum = exp(-(dx * dx + dy * dy + dz * dz) * c.P.inv2l2);
        const double* Li = s.A + pk(i, 0);
        for (int j = 0; j < i; ++j) sum -= Li[j] * V[(int64_t)j * stride];
        const double vi = sum * s.invd[i];
        V[(int64_t)i * stride] = vi;
        acc += vi * vi;
    }
    return fmax(0.0, 1.0 - acc);
}

__global__ void k_solve(SolveCtx c) {
    extern __shared__ double sm[];
    __shared__ int s_w;
    const int tid = threadIdx.x, nt = blockDim.x;
    double* ws_a = c.a_in_smem ? nullptr : c.ws_a + (int64_t)blockIdx.x * c.ws_a_stride;
    Shared s = carve(sm, c.nmax, c.a_in_smem, ws_a);
    double* V = c.ws_v + (int64_t)blockIdx.x * c.ws_v_stride + tid;
    for (;;) {
        if (tid == 0) s_w = atomicAdd(c.counter, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= c.n_work) break;
        const int I = c.order[w];
        const int64_t base = c.b.inst_off[I];
        const int N = (int)(c.b.inst_off[I + 1] - base);
        const int64_t q0 = c.b.q_off[I], q1 = c.b.q_off[I + 1];
        const bool ok = N > 0 && fit_instance(c, s, I, N, base);
        if (c.b.alpha_out)
            for (int j = tid; j < N; j += nt) c.b.alpha_out[base + j] = ok ? s.alpha[j] : NAN;
        for (int64_t p = q0 + tid; p < q1; p += nt) {
            const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
            EvalOut r;
            if (!ok) {
                r.status = N > 0 ? VGP_ST_FACTOR_FAIL : VGP_ST_NO_SUPPORT;
                r.d = INFINITY;
                r.g[0] = r.g[1] = r.g[2] = 0.0;
                r.v = INFINITY;
            } else {
                double xl[3], lo, gro[3];
                query_local(c, I, p, qid, xl);
                if (!(isfinite(xl[0]) && isfinite(xl[1]) && isfinite(xl[2]))) {
                    r.status = VGP_ST_BAD_INPUT;
                    r.d = INFINITY;
                    r.g[0] = r.g[1] = r.g[2] = 0.0;
                    r.v = INFINITY;
                } else {
                    latent_mean(c, s, N, xl, lo, gro);
                    double u = c.b.want_var ? latent_var(c, s, N, xl, V, nt) : 0.0;
                    revert(c.P, lo, gro, u, c.b.want_var != 0, r);
                }
            }
            write_out(c.b, qid, r);
        }
        if (!ok && N > 0 && tid == 0) atomicOr(c.err, kErrFactor);
        __syncthreads();
    }
}

// Backward pass (derived from Eq. 1 and Eq. 3): per instance,
//   obar_q = dL/dd_q * dd/do_q, abar = sum_q obar_q k_q, lambda = A^-1 abar,
//   dL/dx_j = sum_q obar_q alpha_j k_qj (x*_q - x_j) / l^2
//             - sum_i (lambda_i alpha_j + lambda_j alpha_i) k_ij (x_i - x_j) / l^2,
// and dL/dx*_q = dL/dd_q grad d_q.  FP64 throughout.
__global__ void k_backward(SolveCtx c) {
    extern __shared__ double sm[];
    __shared__ int s_w;
    const int tid = threadIdx.x, nt = blockDim.x;
    double* ws_a = c.a_in_smem ? nullptr : c.ws_a + (int64_t)blockIdx.x * c.ws_a_stride;
    Shared s = carve(sm, c.nmax, c.a_in_smem, ws_a);
    const double l2 = c.P.l2;
    for (;;) {
        if (tid == 0) s_w = atomicAdd(c.counter, 1);
        __syncthreads();
        const int w = s_w;
        __syncthreads();
        if (w >= c.n_work) break;
        const int I = c.order[w];
        const int64_t base = c.b.inst_off[I];
        const int N = (int)(c.b.inst_off[I + 1] - base);
        const int64_t q0 = c.b.q_off[I], q1 = c.b.q_off[I + 1];
        SolveCtx cc = c;
        cc.P.precision = VGP_FP64;
        const bool ok = N > 0 && fit_instance(cc, s, I, N, base);
        // per query: obar and dL/dq
        for (int64_t p = q0 + tid; p < q1; p += nt) {
            const int64_t qid = c.b.qidx ? c.b.qidx[p] : p;
            double ob = 0.0, gq[3] = {0.0, 0.0, 0.0};
            if (ok) {
                double xl[3], lo, gro[3];
                query_local(cc, I, p, qid, xl);
                latent_mean(cc, s, N, xl, lo, gro);
                EvalOut r;
                revert(cc.P, lo, gro, 0.0, false, r);
                const double g = c.bw.dL_dd[qid];
                for (int a = 0; a < 3; ++a) gq[a] = g * r.g[a];
                if (r.status == VGP_ST_OK && r.d > 0.0 && lo < 0.0) ob = g * (-l2 / (exp(lo) * r.d));
            }
            c.bw.obar[p] = ob;
            if (c.bw.dL_dq)
                for (int a = 0; a < 3; ++a) c.bw.dL_dq[3 * qid + a] = gq[a];
        }
        __syncthreads();
        if (ok && c.bw.dL_dX) {
            // abar_j and the direct term, thread per training point
            for (int j = tid; j < N; j += nt) {
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
                s.y[j] = 0.0;
                for (int a = 0; a < 3; ++a) g1[a] *= s.alpha[j] / l2;
                const int64_t gi = c.bw.gidx[base + j];
                for (int a = 0; a < 3; ++a) atomicAdd(&c.bw.dL_dX[3 * gi + a], g1[a]);
            }
            __syncthreads();
            // lambda = A^-1 abar (two triangular solves, in place in z -> y)
            const double* A = s.A;
            for (int j = 0; j < N; ++j) {
                const double yj = s.z[j] * s.invd[j];
                for (int i = j + 1 + tid; i < N; i += nt) s.z[i] -= A[pk(i, j)] * yj;
                if (tid == 0) s.y[j] = yj;
                __syncthreads();
            }
            for (int j = N - 1; j >= 0; --j) {
                const double lj = s.y[j] * s.invd[j];
                for (int i = tid; i < j; i += nt) s.y[i] -= A[pk(j, i)] * lj;
                __syncthreads();
                if (tid == 0) s.z[j] = lj;  // z now holds lambda
                __syncthreads();
            }
            for (int j = tid; j < N; j += nt) {
                double g2[3] = {0.0, 0.0, 0.0};
                const double lj = s.z[j], aj = s.alpha[j];
                for (int i = 0; i < N; ++i) {
                    if (i == j) continue;
                    double dx = s.X[3 * i] - s.X[3 * j], dy = s.X[3 * i + 1] - s.X[3 * j + 1],
                           dz = s.X[3 * i + 2] - s.X[3 * j + 2];
                    double k = exp(-(dx * dx + dy * dy + dz * dz) * c.P.inv2l2);
                    double cf = (s.z[i] * aj + lj * s.alpha[i]) * k;
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

// order[] sorted by increasing N via the prefix of the histogram; the kernels walk it from
// the end (largest first) through `rev`.
__global__ void k_order_n(const int64_t* inst_off, int64_t n, int* cursor, int32_t* order) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int N = (int)(inst_off[i + 1] - inst_off[i]);
    int pos = atomicAdd(&cursor[min(N, 1024)], 1);
    order[pos] = (int32_t)i;
}

__global__ void k_reverse_i32(const int32_t* in, int32_t* out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[n - 1 - i];
}

}  // namespace

void solve_batch(const SolveBatch& b, const DevParams& P, int* err_dev, cudaStream_t st, Arena& ar,
                 SolveStats* stats, const BackwardBatch* bw, bool profile) {
    const int64_t n = b.n_inst;
    if (n <= 0) return;
    // size histogram and decreasing-size order
    int* hist = (int*)ar.get(Arena::kHist, sizeof(int) * 2 * 1025, st);
    int* cursor = hist + 1025;
    cudaMemsetAsync(hist, 0, sizeof(int) * 1025, st);
    const int T = 256;
    k_hist_n<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(b.inst_off, n, hist);
    note_launch();
    std::vector<int> h(1025);
    cudaMemcpyAsync(h.data(), hist, sizeof(int) * 1025, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    std::vector<int> start(1026, 0);
    for (int i = 0; i < 1025; ++i) start[i + 1] = start[i] + h[i];
    cudaMemcpyAsync(cursor, start.data(), sizeof(int) * 1025, cudaMemcpyHostToDevice, st);
    int32_t* order_inc = (int32_t*)ar.get(Arena::kOrder, sizeof(int32_t) * 2 * n, st);
    int32_t* order = order_inc + n;
    k_order_n<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(b.inst_off, n, cursor, order_inc);
    note_launch();
    k_reverse_i32<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(order_inc, order, (int)n);
    note_launch();
    if (stats) {
        for (int N = 0; N <= 1024; ++N) {
            int bk = N <= 32 ? 0 : N <= 64 ? 1 : N <= 128 ? 2 : N <= 256 ? 3 : 4;
            stats->bucket_count[bk] += h[N];
            stats->sum_n3 += (double)h[N] * N * N * N;
            stats->sum_n2 += (double)h[N] * N * N;
        }
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (profile) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, st);
    }
    // buckets (descending): [225, 1024] global A; [129, 224], [65, 128], [33, 64], [0, 32] smem A
    struct Bucket { int lo, hi, smem_a, threads; };
    const Bucket buckets[] = {{225, 1024, 0, 256}, {129, 224, 1, 256}, {65, 128, 1, 256},
                              {33, 64, 1, 128}, {0, 32, 1, 64}};
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int* counters = (int*)ar.get(Arena::kCounters, sizeof(int) * 8, st);
    cudaMemsetAsync(counters, 0, sizeof(int) * 8, st);
    int done = 0;  // instances already assigned (from the large end)
    int bi = 0;
    for (const Bucket& bk : buckets) {
        int cnt = 0, nmax = 0;
        for (int N = bk.lo; N <= bk.hi; ++N) {
            cnt += h[N];
            if (h[N]) nmax = N;
        }
        if (cnt == 0) { ++bi; continue; }
        SolveCtx c;
        c.b = b;
        c.P = P;
        c.err = err_dev;
        c.counter = counters + bi;
        c.order = order + done;
        c.n_work = cnt;
        c.nmax = std::max(nmax, 1);
        c.a_in_smem = bk.smem_a;
        c.backward = bw != nullptr;
        if (bw) c.bw = *bw;
        size_t shm = smem_bytes(c.nmax, c.a_in_smem);
        auto kern = bw ? k_backward : k_solve;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bk.threads, shm);
        per_sm = std::max(per_sm, 1);
        int grid = (int)std::min<int64_t>(cnt, (int64_t)n_sm * per_sm);
        c.ws_a_stride = c.a_in_smem ? 0 : pk(c.nmax, 0);
        c.ws_a = c.a_in_smem ? nullptr
                             : (double*)ar.get(Arena::kWs0, sizeof(double) * c.ws_a_stride * grid, st);
        c.ws_v_stride = (int64_t)c.nmax * bk.threads;
        c.ws_v = (b.want_var && !bw) ? (double*)ar.get(Arena::kWs1, sizeof(double) * c.ws_v_stride * grid, st)
                                     : nullptr;
        kern<<<grid, bk.threads, shm, st>>>(c);
        note_launch();
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
}

}  // namespace vgp
