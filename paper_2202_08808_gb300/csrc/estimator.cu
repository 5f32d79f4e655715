// estimator.cu -- training and evaluation of the learned row-size estimator
// (the network is in estimator.cuh), and the features of rows of C.
//
// Training is plain SGD on the mean squared error between the network's
// output and log2(1 + nnz(C_i)), where nnz(C_i) are exact row sizes that the
// library itself produced (the lengths of the rows of C after a build or a
// batch, which are exact symbolic counts).  One step runs four kernels:
//   k_est_fwd       one thread per row: activations, output, loss, dL/do
//   k_est_bwd_rows  one thread per row: dL/dz2, dL/dz1 through the ReLUs
//   k_est_grad      one thread per parameter: sums over the rows
//   k_est_sgd       master <- master - lr * grad; bfloat16 copy for the forward
// Every sum over rows runs in row order in one thread, so a step is
// deterministic.  The forward uses the bfloat16-rounded weights and the
// gradient is taken at them (applied to the float32 master copy).
#include <cuda_bf16.h>

#include <cstring>
#include <string>

#include "estimator.cuh"
#include "internal.h"

using namespace dspg;

namespace {

struct EErr {
    dspg_status st;
    std::string msg;
};

#define ECK(x)                                                                                          \
    do {                                                                                                \
        cudaError_t e_ = (x);                                                                           \
        if (e_ != cudaSuccess) throw EErr{DSPG_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

template <typename T>
void ealloc(T **p, size_t n) {
    if (cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
        cudaGetLastError();
        throw EErr{DSPG_ERR_OOM, "estimator: device allocation failed"};
    }
}

constexpr int EST_NT = 128;
constexpr size_t EST_SMEM = EST_PARAMS * sizeof(float) + 16;

__device__ __forceinline__ void load_weights(float *W, const uint16_t *w) {
    for (int k = threadIdx.x; k < EST_PARAMS; k += blockDim.x) W[k] = bf16_bits_to_float(w[k]);
    __syncthreads();
}

__global__ void __launch_bounds__(EST_NT)
k_est_fwd(const uint16_t *w, const float *X, const float *y, int64_t n, float *H1, float *H2, float *O, float *D,
          double *loss) {
    pdl_begin();
    extern __shared__ __align__(16) float W[];
    load_weights(W, w);
    double part = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        float x[EST_IN];
        for (int c = 0; c < EST_IN; c++) x[c] = X[r * EST_IN + c];
        float h1[EST_HID];
        est_layer1(W, x, h1);
        for (int j = 0; j < EST_HID; j++) H1[r * EST_HID + j] = h1[j];
        float o = W[EST_B3];
        for (int j = 0; j < EST_HID; j++) {
            const float h2 = est_unit2(W, h1, j);
            H2[r * EST_HID + j] = h2;
            o = fmaf(W[EST_W3 + j], h2, o);
        }
        O[r] = o;
        if (y) {
            const float d = o - y[r];
            D[r] = 2.0f * d / (float)n;
            part += (double)d * (double)d;
        }
    }
    if (y) {
        part = warp_sum<double>(part);
        if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(loss, part / (double)n);
    }
}

__global__ void __launch_bounds__(EST_NT)
k_est_bwd_rows(const uint16_t *w, int64_t n, const float *H1, const float *H2, const float *D, float *DZ1,
               float *DZ2) {
    pdl_begin();
    extern __shared__ __align__(16) float W[];
    load_weights(W, w);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const float d = D[r];
        float dz2[EST_HID];
        for (int j = 0; j < EST_HID; j++) {
            dz2[j] = H2[r * EST_HID + j] > 0.0f ? d * W[EST_W3 + j] : 0.0f;
            DZ2[r * EST_HID + j] = dz2[j];
        }
        for (int k = 0; k < EST_HID; k++) {
            float dh = 0.0f;
            for (int j = 0; j < EST_HID; j++) dh = fmaf(dz2[j], W[EST_W2 + j * EST_HID + k], dh);
            DZ1[r * EST_HID + k] = H1[r * EST_HID + k] > 0.0f ? dh : 0.0f;
        }
    }
}

// One thread per parameter, each summing its term over the rows in order.
__global__ void k_est_grad(const float *X, int64_t n, const float *H1, const float *H2, const float *D,
                           const float *DZ1, const float *DZ2, float *grad) {
    pdl_begin();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= EST_PARAMS) return;
    float g = 0.0f;
    if (p < EST_B1) {  // W1[j][c] = sum_r dz1[r][j] x[r][c]
        const int j = p / EST_IN, c = p % EST_IN;
        for (int64_t r = 0; r < n; r++) g = fmaf(DZ1[r * EST_HID + j], X[r * EST_IN + c], g);
    } else if (p < EST_W2) {  // b1[j] = sum_r dz1[r][j]
        const int j = p - EST_B1;
        for (int64_t r = 0; r < n; r++) g += DZ1[r * EST_HID + j];
    } else if (p < EST_B2) {  // W2[j][k] = sum_r dz2[r][j] h1[r][k]
        const int j = (p - EST_W2) / EST_HID, k = (p - EST_W2) % EST_HID;
        for (int64_t r = 0; r < n; r++) g = fmaf(DZ2[r * EST_HID + j], H1[r * EST_HID + k], g);
    } else if (p < EST_W3) {  // b2[j]
        const int j = p - EST_B2;
        for (int64_t r = 0; r < n; r++) g += DZ2[r * EST_HID + j];
    } else if (p < EST_B3) {  // W3[j] = sum_r d[r] h2[r][j]
        const int j = p - EST_W3;
        for (int64_t r = 0; r < n; r++) g = fmaf(D[r], H2[r * EST_HID + j], g);
    } else {  // b3
        for (int64_t r = 0; r < n; r++) g += D[r];
    }
    grad[p] = g;
}

__global__ void k_est_sgd(float *master, const float *grad, float lr, uint16_t *w) {
    pdl_begin();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= EST_PARAMS) return;
    const float v = master[p] - lr * grad[p];
    master[p] = v;
    w[p] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__global__ void k_est_round(const float *master, uint16_t *w) {
    pdl_begin();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < EST_PARAMS) w[p] = __bfloat16_as_ushort(__float2bfloat16_rn(master[p]));
}

// Features of rows (all rows when rows == nullptr) and, when y != nullptr,
// the target log2(1 + len(C_i)).  A row index out of range sets *bad and
// gets zeros.
__global__ void k_row_features(MatView A, MatView B, MatView C, const int32_t *rows, int64_t n, float *X, float *y,
                               unsigned *bad) {
    pdl_begin();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = rows ? rows[t] : (int32_t)t;
        if (i < 0 || i >= A.nrows) {
            atomicOr(bad, 1u);
            for (int c = 0; c < EST_IN; c++) X[t * EST_IN + c] = 0.0f;
            if (y) y[t] = 0.0f;
            continue;
        }
        const int64_t off = A.off[i];
        const int alen = A.len[i];
        long long sum = 0, mx = 0;
        for (int a = 0; a < alen; a++) {
            const long long l = B.len[A.col[off + a]];
            sum += l;
            mx = l > mx ? l : mx;
        }
        float x[EST_IN];
        est_features(x, alen, sum, mx);
        for (int c = 0; c < EST_IN; c++) X[t * EST_IN + c] = x[c];
        if (y) y[t] = log2f(1.0f + (float)C.len[i]);
    }
}

unsigned grid_rows(int64_t n) {
    int64_t g = (n + EST_NT - 1) / EST_NT;
    if (g > 4096) g = 4096;
    return (unsigned)(g < 1 ? 1 : g);
}

void ensure_rows(dspg_estimator *e, int64_t n) {
    if (n <= e->cap) return;
    for (float **p : {&e->H1, &e->H2, &e->DZ1, &e->DZ2}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    for (float **p : {&e->D, &e->O}) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    const int64_t cap = n + n / 2;
    for (float **p : {&e->H1, &e->H2, &e->DZ1, &e->DZ2}) ealloc(p, (size_t)cap * EST_HID);
    for (float **p : {&e->D, &e->O}) ealloc(p, (size_t)cap);
    e->cap = cap;
}

void set_smem_attrs() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(k_est_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EST_SMEM);
    cudaFuncSetAttribute(k_est_bwd_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EST_SMEM);
    done = true;
}

// forward (+ loss and dL/do when y) and, when grad, the backward pass
void run_step(dspg_estimator *e, const float *X, const float *y, int64_t n, bool grad, cudaStream_t s) {
    set_smem_attrs();
    ensure_rows(e, n);
    if (y) ECK(cudaMemsetAsync(e->loss_d, 0, sizeof(double), s));
    launch_k(k_est_fwd, grid_rows(n), EST_NT, EST_SMEM, s, (const uint16_t *)e->w, X, y, n, e->H1, e->H2, e->O, e->D,
             e->loss_d);
    if (!grad) return;
    launch_k(k_est_bwd_rows, grid_rows(n), EST_NT, EST_SMEM, s, (const uint16_t *)e->w, n, (const float *)e->H1,
             (const float *)e->H2, (const float *)e->D, e->DZ1, e->DZ2);
    launch_k(k_est_grad, (EST_PARAMS + 127) / 128, 128, 0, s, X, n, (const float *)e->H1, (const float *)e->H2,
             (const float *)e->D, (const float *)e->DZ1, (const float *)e->DZ2, e->grad);
}

dspg_status efail(dspg_estimator *e, const EErr &x) {
    if (e) e->err = x.msg;
    dspg::set_thread_error(x.msg.c_str());
    return x.st;
}

void check_rows(const float *X, int64_t n) {
    if (n <= 0 || !X) throw EErr{DSPG_ERR_INVALID, "estimator: need n > 0 rows and X"};
}

}  // namespace

void dspg::row_features(const MatView &A, const MatView &B, const MatView &C, const int32_t *rows, int64_t n, float *X,
                        float *y, unsigned *bad, cudaStream_t s) {
    if (n > 0) launch_k(k_row_features, grid_rows(n), EST_NT, 0, s, A, B, C, rows, n, X, y, bad);
}

extern "C" {

dspg_status dspg_estimator_create(dspg_estimator **out, const float *params) {
    dspg_estimator *e = nullptr;
    try {
        if (!out || !params) throw EErr{DSPG_ERR_INVALID, "estimator: out and params must not be NULL"};
        *out = nullptr;
        e = new dspg_estimator();
        ealloc(&e->master, EST_PARAMS);
        ealloc(&e->grad, EST_PARAMS);
        ealloc(&e->w, EST_PARAMS);
        ealloc(&e->loss_d, 1);
        ECK(cudaMemcpy(e->master, params, sizeof(float) * EST_PARAMS, cudaMemcpyHostToDevice));
        ECK(cudaMemset(e->grad, 0, sizeof(float) * EST_PARAMS));
        launch_k(k_est_round, (EST_PARAMS + 127) / 128, 128, 0, (cudaStream_t)0, (const float *)e->master, e->w);
        ECK(cudaGetLastError());
        ECK(cudaDeviceSynchronize());
        *out = e;
        return DSPG_OK;
    } catch (const EErr &x) {
        dspg_status st = efail(nullptr, x);
        dspg_estimator_destroy(e);
        return st;
    }
}

dspg_status dspg_estimator_params(dspg_estimator *e, float *params, void *stream) {
    if (!e || !params) return DSPG_ERR_INVALID;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        ECK(cudaMemcpyAsync(params, e->master, sizeof(float) * EST_PARAMS, cudaMemcpyDeviceToHost, s));
        ECK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const EErr &x) {
        return efail(e, x);
    }
}

dspg_status dspg_estimator_grad(dspg_estimator *e, const float *X, const float *y, int64_t n, float *grad,
                                double *loss, void *stream) {
    if (!e) return DSPG_ERR_INVALID;
    try {
        check_rows(X, n);
        if (!y) throw EErr{DSPG_ERR_INVALID, "estimator: y is NULL"};
        cudaStream_t s = (cudaStream_t)stream;
        run_step(e, X, y, n, true, s);
        if (grad) ECK(cudaMemcpyAsync(grad, e->grad, sizeof(float) * EST_PARAMS, cudaMemcpyDeviceToHost, s));
        if (loss) ECK(cudaMemcpyAsync(loss, e->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s));
        ECK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const EErr &x) {
        return efail(e, x);
    }
}

dspg_status dspg_estimator_train(dspg_estimator *e, const float *X, const float *y, int64_t n, int64_t batch,
                                 int64_t steps, float lr, double *loss, void *stream) {
    if (!e) return DSPG_ERR_INVALID;
    try {
        check_rows(X, n);
        if (!y || batch <= 0 || steps < 0 || !(lr > 0.0f)) throw EErr{DSPG_ERR_INVALID, "estimator: bad training arguments"};
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t nb = (n + batch - 1) / batch;
        for (int64_t k = 0; k < steps; k++) {
            const int64_t b = k % nb;
            const int64_t lo = b * batch, m = (lo + batch <= n) ? batch : n - lo;
            run_step(e, X + lo * EST_IN, y + lo, m, true, s);
            launch_k(k_est_sgd, (EST_PARAMS + 127) / 128, 128, 0, s, e->master, (const float *)e->grad, lr, e->w);
        }
        ECK(cudaGetLastError());
        if (loss) {  // loss of the whole set after training
            run_step(e, X, y, n, false, s);
            ECK(cudaMemcpyAsync(loss, e->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        ECK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const EErr &x) {
        return efail(e, x);
    }
}

dspg_status dspg_estimator_predict(dspg_estimator *e, const float *X, int64_t n, float *out, void *stream) {
    if (!e || !out) return DSPG_ERR_INVALID;
    try {
        check_rows(X, n);
        cudaStream_t s = (cudaStream_t)stream;
        run_step(e, X, nullptr, n, false, s);
        ECK(cudaMemcpyAsync(out, e->O, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        ECK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const EErr &x) {
        return efail(e, x);
    }
}

const char *dspg_estimator_last_error(const dspg_estimator *e) { return e ? e->err.c_str() : dspg_last_error(nullptr); }

void dspg_estimator_destroy(dspg_estimator *e) {
    if (!e) return;
    cudaDeviceSynchronize();
    for (float *p : {e->master, e->grad, e->H1, e->H2, e->D, e->DZ1, e->DZ2, e->O})
        if (p) cudaFree(p);
    if (e->w) cudaFree(e->w);
    if (e->loss_d) cudaFree(e->loss_d);
    delete e;
}

}  // extern "C"
