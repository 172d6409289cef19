// train.cu -- the training-step pieces around the rendering path: the L2 + D-SSIM image loss and
// its gradient (Sec. 3 "Loss Function", App. A.7), a fused Adam update and the sigmoid
// activations of opacities and scales (Sec. 5).
//
// Loss layout: the images are the rs_render outputs, pixel-major and concatenated camera by
// camera (float[P * 3]).  Each CTA owns a 32 x 8 tile of one channel of one image; the
// separable 11 x 11 Gaussian window (sigma 1.5) runs as a horizontal then a vertical pass in
// shared memory over the tile plus a 5-pixel halo (zero outside the image).
//   pass 1: window sums of I, J, I^2, J^2, IJ -> SSIM per pixel (summed per tile for the
//           loss) and App. A.7's E, F, G (written per pixel and channel);
//   pass 2: window sums of E, F, G -> dL/dI = ((1 - lambda) 2 (I - J) - lambda / 2 *
//           ((E*w) + J (F*w) - I (G*w))) / (3 h w n_images);
//   pass 3: one CTA reduces the per-tile partial sums in a fixed order (deterministic).
#include <math.h>
#include <stdint.h>

#include <cmath>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "rs_host.h"
#include "rs_internal.cuh"

namespace rs {

namespace {

constexpr int kR = 5;                   // window radius
constexpr int kTW = 32, kTH = 8;        // output tile
constexpr int kHW = kTW + 2 * kR;       // halo tile width (42)
constexpr int kHH = kTH + 2 * kR;       // halo tile height (18)
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

__constant__ float c_win[2 * kR + 1];   // normalised 1-D Gaussian taps

struct LossImage {
    int W, H;
    int64_t base;        // first pixel of the image
    int tiles_x, tiles_y;
    int part_base;       // first partial-sum slot of the image (tiles_x * tiles_y per channel)
};

struct LossArgs {
    const float* rgb;
    const float* target;
    const LossImage* images;
    int n_images;
    float lambda;
    float* efg;          // per pixel and channel: E, F, G (float[P * 9])
    float2* partial;     // per tile and channel: (sum of SSIM, sum of (I - J)^2)
    float* d_rgb;
    float* loss;
};

__device__ __forceinline__ float load_px(const float* img, const LossImage& im, int x, int y, int stride, int comp) {
    if (x < 0 || y < 0 || x >= im.W || y >= im.H) return 0.f;
    return img[(im.base + (int64_t)y * im.W + x) * stride + comp];
}

// pass 1: statistics, SSIM partial sums, E / F / G
__global__ void __launch_bounds__(256) k_ssim_stats(LossArgs A) {
    const int img = blockIdx.z / 3, ch = blockIdx.z % 3;
    const LossImage im = A.images[img];
    const int tx = blockIdx.x % im.tiles_x, ty = blockIdx.x / im.tiles_x;
    if (ty >= im.tiles_y) return;
    __shared__ float sI[kHH][kHW], sJ[kHH][kHW];
    __shared__ float hs[5][kHH][kTW];
    __shared__ float red[2][256 / 32];
    const int x0 = tx * kTW - kR, y0 = ty * kTH - kR;
    for (int i = threadIdx.x; i < kHH * kHW; i += blockDim.x) {
        const int yy = i / kHW, xx = i % kHW;
        sI[yy][xx] = load_px(A.rgb, im, x0 + xx, y0 + yy, 3, ch);
        sJ[yy][xx] = load_px(A.target, im, x0 + xx, y0 + yy, 3, ch);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHH * kTW; i += blockDim.x) {
        const int yy = i / kTW, xx = i % kTW;
        float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m <= 2 * kR; ++m) {
            const float a = sI[yy][xx + m], b = sJ[yy][xx + m], w = c_win[m];
            s[0] = fmaf(w, a, s[0]);
            s[1] = fmaf(w, b, s[1]);
            s[2] = fmaf(w, a * a, s[2]);
            s[3] = fmaf(w, b * b, s[3]);
            s[4] = fmaf(w, a * b, s[4]);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) hs[k][yy][xx] = s[k];
    }
    __syncthreads();
    const int lx = threadIdx.x % kTW, ly = threadIdx.x / kTW;  // 256 threads = 32 x 8
    const int x = tx * kTW + lx, y = ty * kTH + ly;
    float ssim_v = 0.f, l2_v = 0.f;
    if (x < im.W && y < im.H) {
        float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m <= 2 * kR; ++m) {
            const float w = c_win[m];
#pragma unroll
            for (int k = 0; k < 5; ++k) s[k] = fmaf(w, hs[k][ly + m][lx], s[k]);
        }
        const float mu1 = s[0], mu2 = s[1];
        const float s11 = s[2] - mu1 * mu1, s22 = s[3] - mu2 * mu2, s12 = s[4] - mu1 * mu2;
        const float Av = 2.f * mu1 * mu2 + kC1, Bv = 2.f * s12 + kC2;
        const float Cv = mu1 * mu1 + mu2 * mu2 + kC1, Dv = s11 + s22 + kC2;
        const float CD = Cv * Dv;
        ssim_v = Av * Bv / CD;
        const float k2 = 2.f / (CD * CD);
        float* e = A.efg + ((im.base + (int64_t)y * im.W + x) * 3 + ch) * 3;
        e[0] = k2 * (CD * mu2 * (Bv - Av) - Av * Bv * mu1 * (Dv - Cv));
        e[1] = k2 * Av * CD;
        e[2] = k2 * Av * Bv * Cv;
        const float d = sI[ly + kR][lx + kR] - sJ[ly + kR][lx + kR];
        l2_v = d * d;
    }
    // tile sums (fixed order: warp shuffles, then warps in index order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssim_v += __shfl_xor_sync(0xffffffffu, ssim_v, o);
        l2_v += __shfl_xor_sync(0xffffffffu, l2_v, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = ssim_v;
        red[1][threadIdx.x >> 5] = l2_v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int k = 0; k < 256 / 32; ++k) {
            a += red[0][k];
            b += red[1][k];
        }
        A.partial[(int64_t)(im.part_base + blockIdx.x) * 3 + ch] = make_float2(a, b);
    }
}

// pass 2: window sums of E, F, G and dL/dI
__global__ void __launch_bounds__(256) k_ssim_grad(LossArgs A) {
    const int img = blockIdx.z / 3, ch = blockIdx.z % 3;
    const LossImage im = A.images[img];
    const int tx = blockIdx.x % im.tiles_x, ty = blockIdx.x / im.tiles_x;
    if (ty >= im.tiles_y) return;
    __shared__ float sE[3][kHH][kHW];
    __shared__ float hs[3][kHH][kTW];
    const int x0 = tx * kTW - kR, y0 = ty * kTH - kR;
    for (int i = threadIdx.x; i < kHH * kHW; i += blockDim.x) {
        const int yy = i / kHW, xx = i % kHW;
#pragma unroll
        for (int k = 0; k < 3; ++k) sE[k][yy][xx] = load_px(A.efg, im, x0 + xx, y0 + yy, 9, ch * 3 + k);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHH * kTW; i += blockDim.x) {
        const int yy = i / kTW, xx = i % kTW;
        float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int m = 0; m <= 2 * kR; ++m) {
            const float w = c_win[m];
#pragma unroll
            for (int k = 0; k < 3; ++k) s[k] = fmaf(w, sE[k][yy][xx + m], s[k]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) hs[k][yy][xx] = s[k];
    }
    __syncthreads();
    const int lx = threadIdx.x % kTW, ly = threadIdx.x / kTW;
    const int x = tx * kTW + lx, y = ty * kTH + ly;
    if (x >= im.W || y >= im.H) return;
    float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int m = 0; m <= 2 * kR; ++m) {
        const float w = c_win[m];
#pragma unroll
        for (int k = 0; k < 3; ++k) s[k] = fmaf(w, hs[k][ly + m][lx], s[k]);
    }
    const int64_t p = (im.base + (int64_t)y * im.W + x) * 3 + ch;
    const float I = A.rgb[p], J = A.target[p];
    const float hw = (float)im.W * (float)im.H;
    const float dssim = s[0] + J * s[1] - I * s[2];
    const float g = ((1.f - A.lambda) * 2.f * (I - J) - 0.5f * A.lambda * dssim) / (3.f * hw * (float)A.n_images);
    A.d_rgb[p] = g;
}

// pass 3: the batch loss from the tile partial sums (one CTA, fixed order)
__global__ void k_loss_reduce(LossArgs A) {
    __shared__ double acc[256];
    double local = 0.0;
    for (int img = 0; img < A.n_images; ++img) {
        const LossImage im = A.images[img];
        const int tiles = im.tiles_x * im.tiles_y;
        for (int ch = 0; ch < 3; ++ch) {
            double ss = 0.0, l2 = 0.0;
            for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
                const float2 v = A.partial[(int64_t)(im.part_base + t) * 3 + ch];
                ss += v.x;
                l2 += v.y;
            }
            // block sums in a fixed tree order
            acc[threadIdx.x] = ss;
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if ((int)threadIdx.x < s) acc[threadIdx.x] += acc[threadIdx.x + s];
                __syncthreads();
            }
            const double ssim_sum = acc[0];
            __syncthreads();
            acc[threadIdx.x] = l2;
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if ((int)threadIdx.x < s) acc[threadIdx.x] += acc[threadIdx.x + s];
                __syncthreads();
            }
            const double l2_sum = acc[0];
            __syncthreads();
            const double hw = (double)im.W * im.H;
            local += ((1.0 - A.lambda) * l2_sum / hw + A.lambda * (1.0 - ssim_sum / hw) / 2.0) / 3.0;
        }
    }
    if (threadIdx.x == 0) A.loss[0] = (float)(local / A.n_images);
}

// Adam (Sec. 5): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
    }
}

__global__ void k_sigmoid(const float* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = 1.f / (1.f + expf(-x[i]));
}

__global__ void k_sigmoid_backward(const float* __restrict__ y, const float* __restrict__ dy, float* __restrict__ dx,
                                   int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float yi = y[i];
        dx[i] = dy[i] * yi * (1.f - yi);
    }
}

int elementwise_grid(int64_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(sms, 1) * 8));
}

}  // namespace
}  // namespace rs

using namespace rs;

struct rs_loss_state {
    int device = 0;
    LossImage* images = nullptr;
    int cap_images = 0;
    float* efg = nullptr;
    int64_t cap_efg = 0;
    float2* partial = nullptr;
    int64_t cap_partial = 0;
    bool window_set = false;
};

extern "C" {

rs_status rs_loss_l2_dssim(const float* rgb, const float* target, const rs_camera* cams, int32_t n_cams,
                           float lambda, float* loss_device, float* d_rgb, rs_loss_state** inout,
                           void* cuda_stream) {
    if (!rgb || !target || !loss_device || !d_rgb || !inout)
        return set_error(RS_ERR_INVALID_ARG, "loss: a pointer argument is NULL");
    if (!cams || n_cams < 1) return set_error(RS_ERR_INVALID_ARG, "loss: need at least one image");
    if (!(lambda >= 0.f && lambda <= 1.f)) return set_error(RS_ERR_INVALID_ARG, "loss: lambda must be in [0, 1]");
    std::vector<LossImage> ims((size_t)n_cams);
    int64_t pix = 0;
    int64_t parts = 0;
    int max_tiles = 0;
    for (int c = 0; c < n_cams; ++c) {
        const rs_camera& C = cams[c];
        if (C.width < 1 || C.height < 1 || (int64_t)C.width * C.height >= ((int64_t)1 << 31))
            return set_error(RS_ERR_INVALID_ARG, "loss: image %d has a bad size %dx%d", c, C.width, C.height);
        LossImage& L = ims[(size_t)c];
        L.W = C.width;
        L.H = C.height;
        L.base = pix;
        L.tiles_x = (C.width + kTW - 1) / kTW;
        L.tiles_y = (C.height + kTH - 1) / kTH;
        L.part_base = (int)parts;
        const int tiles = L.tiles_x * L.tiles_y;
        max_tiles = std::max(max_tiles, tiles);
        parts += tiles;
        pix += (int64_t)C.width * C.height;
    }
    if (3 * (int64_t)n_cams > 65535) return set_error(RS_ERR_INVALID_ARG, "loss: at most 21845 images per call");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rs_loss_state* S = *inout;
    if (!S) {
        S = new (std::nothrow) rs_loss_state();
        if (!S) return set_error(RS_ERR_OOM, "host allocation failed");
        cudaGetDevice(&S->device);
        *inout = S;
    }
    auto grow = [&](auto*& ptr, int64_t& cap, int64_t want, size_t elem) -> rs_status {
        if (want <= cap) return RS_OK;
        cap = 0;
        void* q = ptr;
        const rs_status r = device_realloc(&q, elem * (size_t)want);
        ptr = static_cast<std::remove_reference_t<decltype(ptr)>>(q);
        if (r == RS_OK) cap = want;
        return r;
    };
    rs_status st;
    int64_t cap_im = S->cap_images;
    if ((st = grow(S->images, cap_im, n_cams, sizeof(LossImage)))) return st;
    S->cap_images = (int)cap_im;
    if ((st = grow(S->efg, S->cap_efg, pix * 9, sizeof(float)))) return st;
    if ((st = grow(S->partial, S->cap_partial, parts * 3, sizeof(float2)))) return st;
    if (!S->window_set) {
        float w[2 * kR + 1];
        double sum = 0.0;
        for (int m = -kR; m <= kR; ++m) sum += exp(-(double)m * m / (2.0 * 1.5 * 1.5));
        for (int m = -kR; m <= kR; ++m) w[m + kR] = (float)(exp(-(double)m * m / (2.0 * 1.5 * 1.5)) / sum);
        if (cudaMemcpyToSymbol(c_win, w, sizeof(w)) != cudaSuccess) return cuda_check("loss window upload");
        S->window_set = true;
    }
    if (cudaMemcpyAsync(S->images, ims.data(), sizeof(LossImage) * ims.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return cuda_check("loss image table upload");
    LossArgs A{rgb, target, S->images, n_cams, lambda, S->efg, S->partial, d_rgb, loss_device};
    const dim3 grid((unsigned)max_tiles, 1, (unsigned)(3 * n_cams));
    k_ssim_stats<<<grid, 256, 0, s>>>(A);
    k_ssim_grad<<<grid, 256, 0, s>>>(A);
    k_loss_reduce<<<1, 256, 0, s>>>(A);
    return cuda_check("loss launch");
}

rs_status rs_loss_state_destroy(rs_loss_state* S) {
    if (!S) return RS_OK;
    cudaDeviceSynchronize();
    if (S->images) cudaFree(S->images);
    if (S->efg) cudaFree(S->efg);
    if (S->partial) cudaFree(S->partial);
    delete S;
    return cuda_check("rs_loss_state_destroy");
}

rs_status rs_adam_step(float* params, const float* grads, float* m, float* v, int64_t count, float lr, float beta1,
                       float beta2, float eps, int32_t step, void* cuda_stream) {
    if (count < 0 || (count > 0 && (!params || !grads || !m || !v)))
        return set_error(RS_ERR_INVALID_ARG, "adam: bad buffers");
    if (step < 1) return set_error(RS_ERR_INVALID_ARG, "adam: step must be >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) || !std::isfinite(lr))
        return set_error(RS_ERR_INVALID_ARG, "adam: bad hyper-parameters");
    if (count == 0) return RS_OK;
    const float bc1 = (float)(1.0 / (1.0 - pow((double)beta1, step)));
    const float bc2 = (float)(1.0 / (1.0 - pow((double)beta2, step)));
    k_adam<<<elementwise_grid(count), 256, 0, (cudaStream_t)cuda_stream>>>(params, grads, m, v, count, lr, beta1,
                                                                           beta2, eps, bc1, bc2);
    return cuda_check("adam launch");
}

rs_status rs_sigmoid(const float* x, float* y, int64_t count, void* cuda_stream) {
    if (count < 0 || (count > 0 && (!x || !y))) return set_error(RS_ERR_INVALID_ARG, "sigmoid: bad buffers");
    if (count == 0) return RS_OK;
    k_sigmoid<<<elementwise_grid(count), 256, 0, (cudaStream_t)cuda_stream>>>(x, y, count);
    return cuda_check("sigmoid launch");
}

rs_status rs_sigmoid_backward(const float* y, const float* dy, float* dx, int64_t count, void* cuda_stream) {
    if (count < 0 || (count > 0 && (!y || !dy || !dx)))
        return set_error(RS_ERR_INVALID_ARG, "sigmoid backward: bad buffers");
    if (count == 0) return RS_OK;
    k_sigmoid_backward<<<elementwise_grid(count), 256, 0, (cudaStream_t)cuda_stream>>>(y, dy, dx, count);
    return cuda_check("sigmoid backward launch");
}

}  // extern "C"
