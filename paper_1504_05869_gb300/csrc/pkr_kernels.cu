// pkr_kernels.cu -- source preparation (step a0) and the deterministic
// binary64 reductions of the solver.
//
// Source (text after Eq. poisson1): S = (rho - <rho>) c_s^2 (tau_lb - 1/2)/eps.
// The mean is a two-pass reduction in a fixed order (per-thread strided sums,
// a fixed shuffle tree per block, then one block over the block partials), so
// repeated runs give bit-identical S.
#include <cuda_runtime.h>

#include <cstddef>

#include <cuda_fp16.h>

#include "pkr_internal.h"

namespace pkr {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(kRedThreads)
rho_partials_kernel(const double* __restrict__ rho, int64_t V, double* __restrict__ partials,
                    int* nonfinite)
{
    __shared__ double sm[kRedThreads / 32];
    double acc = 0.0;
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride) {
        const double r = rho[i];
        bad |= !isfinite(r);
        acc += r;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(nonfinite, 1);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) t += sm[k];
        partials[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kRedThreads)
finalize_mean_kernel(const double* __restrict__ partials, int n, int64_t V, double* mean)
{
    __shared__ double sm[kRedThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kRedThreads) acc += partials[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) t += sm[k];
        *mean = t / (double)V;
    }
}

template <typename T>
__global__ void make_source_kernel(const double* __restrict__ rho, const double* __restrict__ mean,
                                   double scale, int64_t V, T* __restrict__ S)
{
    const double m = *mean;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride)
        S[i] = (T)((rho[i] - m) * scale);
}

// out4[0] = max |dPhi|, out4[1] = ||dPhi||_2 / ||Phi||_2 (0 if both vanish,
// +inf if only Phi does), out4[2] = ||Phi||_2, out4[3] = sum Phi (the mass).
// One block of kRedThreads; out4 is complete when thread 0 returns.
__device__ __forceinline__ void finalize_block(const double* __restrict__ partials, int n,
                                               double* out4, double* v4 = nullptr)
{
    __shared__ double s0[kRedThreads / 32], s1[kRedThreads / 32], s2[kRedThreads / 32],
        s3[kRedThreads / 32];
    double d2 = 0.0, n2 = 0.0, mx = 0.0, ms = 0.0;
    for (int i = threadIdx.x; i < n; i += kRedThreads) {
        d2 += partials[4 * i + 0];
        n2 += partials[4 * i + 1];
        mx = fmax(mx, partials[4 * i + 2]);
        ms += partials[4 * i + 3];
    }
    d2 = warp_sum(d2);
    n2 = warp_sum(n2);
    mx = warp_max(mx);
    ms = warp_sum(ms);
    if ((threadIdx.x & 31) == 0) {
        s0[threadIdx.x >> 5] = d2;
        s1[threadIdx.x >> 5] = n2;
        s2[threadIdx.x >> 5] = mx;
        s3[threadIdx.x >> 5] = ms;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) {
            a += s0[k];
            b += s1[k];
            c = fmax(c, s2[k]);
            d += s3[k];
        }
        out4[0] = c;
        out4[1] = (b > 0.0) ? sqrt(a) / sqrt(b) : (a == 0.0 ? 0.0 : INFINITY);
        out4[2] = sqrt(b);
        out4[3] = d;
        // a NaN anywhere poisons the max; report it
        if (!(a == a) || !(b == b)) {
            out4[0] = NAN;
            out4[1] = NAN;
        }
        if (v4) {   // the same values, in registers of thread 0
            const bool bad = !(a == a) || !(b == b);
            v4[0] = bad ? NAN : c;
            v4[1] = bad ? NAN : ((b > 0.0) ? sqrt(a) / sqrt(b) : (a == 0.0 ? 0.0 : INFINITY));
            v4[2] = sqrt(b);
            v4[3] = d;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads)
finalize_residual_kernel(const double* __restrict__ partials, int n, double* out4)
{
    finalize_block(partials, n, out4);
}

// finalize_residual followed, in thread 0, by the stopping rule of
// pkr_plan_run applied on the device (check step j of a captured run).
// Non-finite out4[0] or out4[2], or growth by 1e6 over the smallest residual
// after two checks, stop with PKR_EDIVERGED; a residual below tol stops with
// PKR_OK.  Once stopped it does nothing.
__global__ void __launch_bounds__(kRedThreads)
finalize_check_kernel(const double* __restrict__ partials, int n, double* out4, RunCtl* ctl,
                      double tol, int tol_kind, int j)
{
    if (ctl->stop) return;
    // thread 0 reads the rule's state while the block reduces
    int nc = 0;
    double min_res = 0.0;
    if (threadIdx.x == 0) {
        nc = ctl->nchecks + 1;
        min_res = ctl->min_res;
    }
    double v4[4];
    finalize_block(partials, n, out4, v4);
    if (threadIdx.x != 0) return;
    const double r = v4[tol_kind == PKR_TOL_MAX_ABS_DPHI ? 0 : 1];
    RunCtl o = *ctl;
    o.last_res = r;
    o.nchecks = nc;
    if (!isfinite(v4[0]) || !isfinite(v4[2]) || (nc > 2 && r > 1e6 * min_res && r > 1e-300)) {
        o.status = PKR_EDIVERGED;
        o.stop = 1;
        o.done_at = j;
    } else {
        if (r < min_res) o.min_res = r;
        if (tol > 0.0 && r < tol) {
            o.status = PKR_OK;
            o.stop = 1;
            o.done_at = j;
        }
    }
    *ctl = o;
}

// Per-grid residual of a batch check step: sums the grid's tile partials in
// tile order (deterministic), one block per grid.
__global__ void __launch_bounds__(kRedThreads)
batch_reduce_kernel(const BatchState* st, int stride_bytes)
{
    const int g = blockIdx.x;
    if (g >= st->ngrids) return;
    const unsigned char* base = static_cast<const unsigned char*>(st->grids);
    const size_t off = offsetof(BatchGrid<double>, tile_begin);
    const int tb = *reinterpret_cast<const int*>(base + (size_t)g * stride_bytes + off);
    const int te = (g + 1 < st->ngrids)
                       ? *reinterpret_cast<const int*>(base + (size_t)(g + 1) * stride_bytes + off)
                       : st->ntiles;
    const double* p = st->tile_partials;
    __shared__ double s0[kRedThreads / 32], s1[kRedThreads / 32], s2[kRedThreads / 32],
        s3[kRedThreads / 32];
    double d2 = 0.0, n2 = 0.0, mx = 0.0, ms = 0.0;
    for (int t = tb + (int)threadIdx.x; t < te; t += kRedThreads) {
        d2 += p[4 * (int64_t)t + 0];
        n2 += p[4 * (int64_t)t + 1];
        mx = fmax(mx, p[4 * (int64_t)t + 2]);
        ms += p[4 * (int64_t)t + 3];
    }
    d2 = warp_sum(d2);
    n2 = warp_sum(n2);
    mx = warp_max(mx);
    ms = warp_sum(ms);
    if ((threadIdx.x & 31) == 0) {
        s0[threadIdx.x >> 5] = d2;
        s1[threadIdx.x >> 5] = n2;
        s2[threadIdx.x >> 5] = mx;
        s3[threadIdx.x >> 5] = ms;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) {
            a += s0[k];
            b += s1[k];
            c = fmax(c, s2[k]);
            d += s3[k];
        }
        double* out = st->grid_res + 4 * g;
        out[0] = c;
        out[1] = (b > 0.0) ? sqrt(a) / sqrt(b) : (a == 0.0 ? 0.0 : INFINITY);
        out[2] = sqrt(b);
        out[3] = d;
        if (!(a == a) || !(b == b)) {
            out[0] = NAN;
            out[1] = NAN;
        }
        // binary32 grids: the next step removes the measured mass through
        // its source (sum_i chi_i = 1, so -mass / V per site removes it)
        const BatchGrid<double>& gd =
            *reinterpret_cast<const BatchGrid<double>*>(base + (size_t)g * stride_bytes);
        if (gd.soff) *gd.soff = isfinite(d) ? -d / (double)gd.V : 0.0;
    }
}

__global__ void batch_step_increment_kernel(BatchState* st) { st->step += 1; }

// Storage conversion with a per-plane shift: out[i*V + x] = in[i*V + x] - sh[i]
// (binary16 input: scaled by *scale first).
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(__half v) { return (double)__half2float(v); }

template <typename TI, typename TO>
__global__ void convert_shift_kernel(const TI* __restrict__ in, TO* __restrict__ out, int Q,
                                     int64_t V, const double* __restrict__ sh,
                                     const float* __restrict__ scale)
{
    const int64_t n = (int64_t)Q * V;
    const double sc = scale ? (double)*scale : 1.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        out[k] = (TO)(to_double(in[k]) * sc - sh[k / V]);
}

// max |in * scale - sh_i| over Q planes, as binary64 bits (atomicMax into *out).
template <typename TI>
__global__ void absmax_shift_kernel(const TI* __restrict__ in, int Q, int64_t V,
                                    const double* __restrict__ sh,
                                    const float* __restrict__ scale, unsigned long long* out)
{
    const int64_t n = (int64_t)Q * V;
    const double sc = scale ? (double)*scale : 1.0;
    double m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        m = fmax(m, fabs(to_double(in[k]) * sc - sh[k / V]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// 64-bit fixed point: out = round((in * scale - sh_i) 2^F).
template <typename TI>
__global__ void convert_fx_kernel(const TI* __restrict__ in, long long* __restrict__ out, int Q,
                                  int64_t V, const double* __restrict__ sh,
                                  const float* __restrict__ scale, int F)
{
    const int64_t n = (int64_t)Q * V;
    const double sc = scale ? (double)*scale : 1.0;
    const double f = ldexp(1.0, F);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        out[k] = __double2ll_rn((to_double(in[k]) * sc - sh[k / V]) * f);
}

__global__ void h16_rescale_kernel(float* sc, unsigned int* pmax, int next)
{
    const float m = __uint_as_float(*pmax);
    if (m > 0.f && isfinite(m)) {
        // smallest power of two s with 4 m / s <= 65504
        int e = 0;
        frexpf(4.0f * m / 65504.0f, &e);
        sc[next] = ldexpf(1.0f, e);
    }
    *pmax = 0u;
}

__global__ void fx_rescale_kernel(int* F, unsigned long long* fmax, int next)
{
    const unsigned long long m = *fmax;
    int sh = 0;
    if (m > (1ull << 54)) sh = (64 - __clzll((long long)m)) - 52;
    F[next] = F[next ^ 1] - sh;
    *fmax = 0ull;
}

__global__ void absmax_f64_kernel(const double* __restrict__ S, int64_t V,
                                  unsigned long long* out)
{
    double m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride)
        m = fmax(m, fabs(S[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void absmax_f32_kernel(const float* __restrict__ S, int64_t V, unsigned int* out)
{
    float m = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += stride)
        m = fmaxf(m, fabsf(S[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Population storage conversion (binary32 -> binary64 or back), n elements.
template <typename TI, typename TO>
__global__ void convert_kernel(const TI* __restrict__ in, TO* __restrict__ out, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (TO)in[i];
}

}  // namespace

int launch_batch_reduce(BatchState* state, int max_grids, int grid_stride_bytes, void* stream)
{
    batch_reduce_kernel<<<max_grids, kRedThreads, 0, (cudaStream_t)stream>>>(state,
                                                                             grid_stride_bytes);
    return (int)cudaGetLastError();
}

// One thread per grid of a 64-bit fixed-point batch, after the step and
// before the step counter moves: the array the grid read this step (parity
// of its age) is the one its next step writes; set its exponent from the
// bit length of this step's largest |stored| and reset the bound.
__global__ void batch_fx_rescale_kernel(const BatchState* st)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= st->ngrids) return;
    const BatchGrid<double>& gd = static_cast<const BatchGrid<double>*>(st->grids)[g];
    const int cur = (int)((st->step - gd.join) & 1);
    const unsigned long long m = *gd.fxmax;
    int sh = 0;
    if (m > (1ull << 54)) sh = (64 - __clzll((long long)m)) - 52;
    gd.fxF[cur] = gd.fxF[cur ^ 1] - sh;
    *gd.fxmax = 0ull;
}

int launch_batch_fx_rescale(BatchState* state, int max_grids, void* stream)
{
    batch_fx_rescale_kernel<<<(max_grids + 127) / 128, 128, 0, (cudaStream_t)stream>>>(state);
    return (int)cudaGetLastError();
}

int launch_batch_increment(BatchState* state, void* stream)
{
    batch_step_increment_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(state);
    return (int)cudaGetLastError();
}

int launch_convert(const void* in, int in_precision, void* out, int out_precision, int64_t n,
                   void* stream)
{
    const int blocks = 152 * 16;
    cudaStream_t st = (cudaStream_t)stream;
    if (in_precision == PKR_FP32 && out_precision == PKR_FP64)
        convert_kernel<float, double><<<blocks, 256, 0, st>>>(static_cast<const float*>(in),
                                                              static_cast<double*>(out), n);
    else if (in_precision == PKR_FP64 && out_precision == PKR_FP32)
        convert_kernel<double, float><<<blocks, 256, 0, st>>>(static_cast<const double*>(in),
                                                              static_cast<float*>(out), n);
    else if (in_precision == out_precision)
        return (int)cudaMemcpyAsync(out, in, (size_t)n * (in_precision == PKR_FP64 ? 8 : 4),
                                    cudaMemcpyDeviceToDevice, st);
    else
        return (int)cudaErrorInvalidValue;
    return (int)cudaGetLastError();
}

int launch_convert_shift(const void* in, int in_precision, void* out, int out_precision, int Q,
                         int64_t V, const double* shift, void* stream, const float* in_scale)
{
    const int blocks = 152 * 16;
    cudaStream_t st = (cudaStream_t)stream;
    const float* sc = in_precision == kFP16 ? in_scale : nullptr;
    if (in_precision == kFP16 && !sc) return (int)cudaErrorInvalidValue;
#define PKR_CONV(TI, TO)                                                                     \
    convert_shift_kernel<TI, TO><<<blocks, 256, 0, st>>>(static_cast<const TI*>(in),         \
                                                         static_cast<TO*>(out), Q, V, shift, sc)
    if (out_precision == PKR_FP64) {
        if (in_precision == PKR_FP64) PKR_CONV(double, double);
        else if (in_precision == PKR_FP32) PKR_CONV(float, double);
        else if (in_precision == kFP16) PKR_CONV(__half, double);
        else return (int)cudaErrorInvalidValue;
    } else if (out_precision == PKR_FP32) {
        if (in_precision == PKR_FP64) PKR_CONV(double, float);
        else if (in_precision == PKR_FP32) PKR_CONV(float, float);
        else if (in_precision == kFP16) PKR_CONV(__half, float);
        else return (int)cudaErrorInvalidValue;
    } else {
        return (int)cudaErrorInvalidValue;
    }
#undef PKR_CONV
    return (int)cudaGetLastError();
}

int launch_h16_rescale(float* sc, unsigned int* pmax, int next, void* stream)
{
    h16_rescale_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(sc, pmax, next);
    return (int)cudaGetLastError();
}

int launch_fx_rescale(int* F, unsigned long long* fmax, int next, void* stream)
{
    fx_rescale_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(F, fmax, next);
    return (int)cudaGetLastError();
}

int launch_absmax_f64(const double* S, int64_t V, unsigned long long* out, void* stream)
{
    int blocks = (int)((V + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    absmax_f64_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(S, V, out);
    return (int)cudaGetLastError();
}

int launch_absmax_f32(const float* S, int64_t V, unsigned int* out, void* stream)
{
    int blocks = (int)((V + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    absmax_f32_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(S, V, out);
    return (int)cudaGetLastError();
}

int launch_rho_partials(const double* rho, int64_t V, double* partials, int nblocks,
                        int* nonfinite, void* stream)
{
    rho_partials_kernel<<<nblocks, kRedThreads, 0, (cudaStream_t)stream>>>(rho, V, partials,
                                                                           nonfinite);
    return (int)cudaGetLastError();
}

int launch_finalize_mean(const double* partials, int nblocks, int64_t V, double* mean,
                         void* stream)
{
    finalize_mean_kernel<<<1, kRedThreads, 0, (cudaStream_t)stream>>>(partials, nblocks, V, mean);
    return (int)cudaGetLastError();
}

int launch_make_source(const double* rho, const double* mean, double scale, int64_t V, void* S,
                       int precision, void* stream)
{
    int blocks = (int)((V + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (precision == PKR_FP64)
        make_source_kernel<double><<<blocks, 256, 0, (cudaStream_t)stream>>>(
            rho, mean, scale, V, static_cast<double*>(S));
    else
        make_source_kernel<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(
            rho, mean, scale, V, static_cast<float*>(S));
    return (int)cudaGetLastError();
}

int launch_finalize_residual(const double* partials, int nblocks, double* out4, void* stream)
{
    finalize_residual_kernel<<<1, kRedThreads, 0, (cudaStream_t)stream>>>(partials, nblocks, out4);
    return (int)cudaGetLastError();
}

int launch_finalize_check(const double* partials, int nblocks, double* out4, RunCtl* ctl,
                          double tol, int tol_kind, int j, void* stream)
{
    finalize_check_kernel<<<1, kRedThreads, 0, (cudaStream_t)stream>>>(partials, nblocks, out4,
                                                                       ctl, tol, tol_kind, j);
    return (int)cudaGetLastError();
}

int launch_absmax_shift(const void* in, int in_precision, int Q, int64_t V, const double* shift,
                        const float* in_scale, unsigned long long* out, void* stream)
{
    const int blocks = 152 * 8;
    cudaStream_t st = (cudaStream_t)stream;
    if (in_precision == PKR_FP64)
        absmax_shift_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(in), Q, V,
                                                            shift, nullptr, out);
    else if (in_precision == PKR_FP32)
        absmax_shift_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(in), Q, V,
                                                           shift, nullptr, out);
    else if (in_precision == kFP16 && in_scale)
        absmax_shift_kernel<__half><<<blocks, 256, 0, st>>>(static_cast<const __half*>(in), Q, V,
                                                            shift, in_scale, out);
    else
        return (int)cudaErrorInvalidValue;
    return (int)cudaGetLastError();
}

int launch_convert_fx(const void* in, int in_precision, long long* out, int Q, int64_t V,
                      const double* shift, const float* in_scale, int F, void* stream)
{
    const int blocks = 152 * 16;
    cudaStream_t st = (cudaStream_t)stream;
    if (in_precision == PKR_FP64)
        convert_fx_kernel<double><<<blocks, 256, 0, st>>>(static_cast<const double*>(in), out, Q,
                                                          V, shift, nullptr, F);
    else if (in_precision == PKR_FP32)
        convert_fx_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(in), out, Q, V,
                                                         shift, nullptr, F);
    else if (in_precision == kFP16 && in_scale)
        convert_fx_kernel<__half><<<blocks, 256, 0, st>>>(static_cast<const __half*>(in), out, Q,
                                                          V, shift, in_scale, F);
    else
        return (int)cudaErrorInvalidValue;
    return (int)cudaGetLastError();
}

}  // namespace pkr
