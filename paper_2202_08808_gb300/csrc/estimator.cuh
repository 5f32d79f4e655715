// estimator.cuh -- the learned row-size estimator's network, shared by the
// training kernels (estimator.cu) and the sizing pass (spgemm.cu).
//
// The paper sizes rows by nothing but Gustavson's recompute (Section 6.1);
// this estimator is an addition of the library.  For a row i of C = A B it
// predicts o = log2(1 + nnz(C_i)) from four features,
//   x = log2(1 + [len(A_i), sum_k len(B_k), max_k len(B_k), mean_k len(B_k)]),
// through x -> 64 ReLU -> 64 ReLU -> 1.  Parameters are one flat vector:
// W1 (64 x 4, row-major), b1 (64), W2 (64 x 64, row-major), b2 (64),
// W3 (64), b3 (1): EST_PARAMS numbers.  The network computes with its
// weights rounded to bfloat16 and accumulates in float32.
#pragma once

#include <stdint.h>

namespace dspg {

constexpr int EST_IN = 4;
constexpr int EST_HID = 64;
constexpr int EST_W1 = 0;
constexpr int EST_B1 = EST_W1 + EST_HID * EST_IN;
constexpr int EST_W2 = EST_B1 + EST_HID;
constexpr int EST_B2 = EST_W2 + EST_HID * EST_HID;
constexpr int EST_W3 = EST_B2 + EST_HID;
constexpr int EST_B3 = EST_W3 + EST_HID;
constexpr int EST_PARAMS = EST_B3 + 1;  // 4545

#ifdef __CUDACC__

// bfloat16 bits -> float (exact: a bfloat16 is the top half of a float).
__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// The four inputs from len(A_i), the sum and the maximum of the B-row lengths.
__device__ __forceinline__ void est_features(float x[EST_IN], long long alen, long long bsum, long long bmax) {
    x[0] = log2f(1.0f + (float)alen);
    x[1] = log2f(1.0f + (float)bsum);
    x[2] = log2f(1.0f + (float)bmax);
    x[3] = log2f(1.0f + (alen > 0 ? (float)((double)bsum / (double)alen) : 0.0f));
}

// First layer: h1 = relu(W1 x + b1).  W is the float copy of the weights
// (shared memory), in the flat layout above.
__device__ __forceinline__ void est_layer1(const float *W, const float x[EST_IN], float h1[EST_HID]) {
#pragma unroll
    for (int j = 0; j < EST_HID; j++) {
        float z = W[EST_B1 + j];
#pragma unroll
        for (int c = 0; c < EST_IN; c++) z = fmaf(W[EST_W1 + j * EST_IN + c], x[c], z);
        h1[j] = fmaxf(z, 0.0f);
    }
}

// Second layer unit j: relu(W2[j,:] h1 + b2[j]).
__device__ __forceinline__ float est_unit2(const float *W, const float h1[EST_HID], int j) {
    float z = W[EST_B2 + j];
    const float4 *w4 = reinterpret_cast<const float4 *>(W + EST_W2 + j * EST_HID);
#pragma unroll
    for (int k = 0; k < EST_HID / 4; k++) {
        const float4 w = w4[k];
        z = fmaf(w.x, h1[4 * k], z);
        z = fmaf(w.y, h1[4 * k + 1], z);
        z = fmaf(w.z, h1[4 * k + 2], z);
        z = fmaf(w.w, h1[4 * k + 3], z);
    }
    return fmaxf(z, 0.0f);
}

// The network's output for one row.
__device__ __forceinline__ float est_forward(const float *W, const float x[EST_IN]) {
    float h1[EST_HID];
    est_layer1(W, x, h1);
    float o = W[EST_B3];
    for (int j = 0; j < EST_HID; j++) o = fmaf(W[EST_W3 + j], est_unit2(W, h1, j), o);
    return o;
}

#endif  // __CUDACC__

}  // namespace dspg
