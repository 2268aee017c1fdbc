// spectra.cu -- pseudo-C_l, shot noise, field combination, bandpower binning
// and their vector-Jacobian products (arXiv:2312.12285, Sec. 2.1).
//
// All sums run in FP64 in a fixed order (deterministic); none of these
// kernels is on the O(N lmax^2) path.
#include "common.cuh"

#include <math_constants.h>

namespace psht {

__device__ __forceinline__ void pair_of(int p, int nf, int& f, int& g) {
    // p = f*nf - f(f-1)/2 + (g - f), f <= g
    int base = 0;
    f = 0;
    while (base + (nf - f) <= p) {
        base += nf - f;
        ++f;
    }
    g = f + (p - base);
}

// C_l^{fg} = [Re(a_l0 conj b_l0) + 2 sum_{m>=1} Re(a_lm conj b_lm)]/(2l+1) - N^{fg}
// (Eq. pseudoCl with a_{l,-m} = (-1)^m conj(a_lm) for real weights).
__global__ void cl_kernel(int L, const double2* __restrict__ alm, int nf, const double* __restrict__ noise,
                          double* __restrict__ out) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int p = blockIdx.y;
    if (l > L) return;
    int f, g;
    pair_of(p, nf, f, g);
    const int64_t M = (int64_t)(L + 1) * (L + 2) / 2;
    const double2* a = alm + (int64_t)f * M;
    const double2* b = alm + (int64_t)g * M;
    double s0 = 0.0, s = 0.0;
    {
        const double2 u = a[l], v = b[l];
        s0 = u.x * v.x + u.y * v.y;
    }
    for (int m = 1; m <= l; ++m) {
        const int64_t idx = tri_base(m, L) + l;
        const double2 u = a[idx], v = b[idx];
        s += u.x * v.x + u.y * v.y;
    }
    double c = (s0 + 2.0 * s) / (2.0 * l + 1.0);
    if (noise) c -= noise[f * nf + g];
    out[(int64_t)p * (L + 1) + l] = c;
}

// grad_a^f(l,m) = c_m/(2l+1) sum_g S^{fg}_l a^g(l,m),  S^{fg} = G^{p(f,g)} (f != g), 2 G^{p(f,f)}.
__global__ void cl_backward_kernel(int L, const double2* __restrict__ alm, int nf, const double* __restrict__ gcl,
                                   double2* __restrict__ galm) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    const int f = blockIdx.z;
    if (l > L || l < m) return;
    const int64_t M = (int64_t)(L + 1) * (L + 2) / 2;
    const int64_t idx = tri_base(m, L) + l;
    const double cm = (m == 0 ? 1.0 : 2.0) / (2.0 * l + 1.0);
    double re = 0.0, im = 0.0;
    for (int g = 0; g < nf; ++g) {
        const int lo = f < g ? f : g, hi = f < g ? g : f;
        const int p = lo * nf - lo * (lo - 1) / 2 + (hi - lo);
        double s = gcl[(int64_t)p * (L + 1) + l];
        if (g == f) s *= 2.0;
        const double2 v = alm[(int64_t)g * M + idx];
        re += s * v.x;
        im += s * v.y;
    }
    galm[(int64_t)f * M + idx] = make_double2(cm * re, cm * im);
}

__global__ void noise_grad_kernel(int L, int nf, const double* __restrict__ gcl, double* __restrict__ gnoise) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf * nf) return;
    const int f = t / nf, g = t % nf;
    double s = 0.0;
    if (f <= g) {
        const int p = f * nf - f * (f - 1) / 2 + (g - f);
        for (int l = 0; l <= L; ++l) s -= gcl[(int64_t)p * (L + 1) + l];
    }
    gnoise[t] = s;
}

// Bandpowers C_b = sum_l theta_b^l C_l, theta = 1/Delta_l on [e_b, e_{b+1}) (Sec. 2.1).
// Bin edges are clamped into [0, L+1] and made non-decreasing on the device,
// so a malformed edge array cannot send a read or write outside the spectra.
__device__ __forceinline__ void bin_edges(const int* __restrict__ edges, int b, int L, int& lo, int& hi) {
    lo = min(max(edges[b], 0), L + 1);
    hi = min(max(edges[b + 1], lo), L + 1);
}

__global__ void bin_kernel(int L, const double* __restrict__ cl, int nspec, const int* __restrict__ edges,
                           int nbin, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nspec * nbin) return;
    const int s = t / nbin, b = t % nbin;
    int lo, hi;
    bin_edges(edges, b, L, lo, hi);
    double acc = 0.0;
    for (int l = lo; l < hi; ++l) acc += cl[(int64_t)s * (L + 1) + l];
    out[t] = hi > lo ? acc / (double)(hi - lo) : 0.0;
}

__global__ void bin_backward_kernel(int L, const double* __restrict__ gb, int nspec, const int* __restrict__ edges,
                                    int nbin, double* __restrict__ gcl) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nspec * (L + 1)) return;
    const int s = t / (L + 1), l = t % (L + 1);
    double v = 0.0;
    for (int b = 0; b < nbin; ++b) {
        int lo, hi;
        bin_edges(edges, b, L, lo, hi);
        if (l >= lo && l < hi) v += gb[(int64_t)s * nbin + b] / (double)(hi - lo);
    }
    gcl[t] = v;
}

// alm_out[o] = sum_s coef[o][s] alm_src[s]
__global__ void combine_kernel(int64_t M, const double2* __restrict__ src, int nsrc, const double* __restrict__ coef,
                               int nout, double2* __restrict__ out) {
    const int64_t total = (int64_t)nout * M;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(t / M);
        const int64_t idx = t - (int64_t)o * M;
        double re = 0.0, im = 0.0;
        for (int s = 0; s < nsrc; ++s) {
            const double c = coef[o * nsrc + s];
            const double2 v = src[(int64_t)s * M + idx];
            re += c * v.x;
            im += c * v.y;
        }
        out[t] = make_double2(re, im);
    }
}

__global__ void combine_noise_kernel(const double* __restrict__ nsrc_v, int nsrc, const double* __restrict__ coef,
                                     int nout, double* __restrict__ nout_v) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nout * nout) return;
    const int o = t / nout, q = t % nout;
    double s = 0.0;  // N_out = C N_src C^T
    for (int k = 0; k < nsrc; ++k)
        for (int j = 0; j < nsrc; ++j) s += coef[o * nsrc + k] * coef[q * nsrc + j] * nsrc_v[k * nsrc + j];
    nout_v[t] = s;
}

// Shot noise: per-catalog block partials of sum w^2 (fixed partition), then a
// fixed-order sum per field.
template <typename T>
__global__ void sumsq_kernel(const __grid_constant__ PrepParams p, double* __restrict__ partial, int nblk) {
    const int c = blockIdx.y;
    const CatDesc& cd = p.cat[c];
    const T* w = static_cast<const T*>(cd.w);
    const int64_t per = (cd.n + nblk - 1) / nblk;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(cd.n, i0 + per);
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double v = (double)w[i];
        s += v * v;
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)c * nblk + blockIdx.x] = red[0];
}

__global__ void noise_final_kernel(const __grid_constant__ PrepParams p, const double* __restrict__ partial, int nblk,
                                   double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.nfield * p.nfield) return;
    const int f = t / p.nfield, g = t % p.nfield;
    if (f != g) {
        out[t] = 0.0;
        return;
    }
    double tot = 0.0;
    for (int c = 0; c < p.ncat; ++c) {
        if (p.cat[c].field != f) continue;
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[(int64_t)c * nblk + b];
        tot += p.cat[c].coeff * p.cat[c].coeff * s;
    }
    out[t] = tot / (4.0 * CUDART_PI);
}

// ------------------------------------------------------------ launchers --
cudaError_t launch_cl(int L, const double* alm, int nf, const double* noise, double* out, cudaStream_t st) {
    const int npair = nf * (nf + 1) / 2;
    dim3 grid((L + 1 + 127) / 128, npair);
    cl_kernel<<<grid, 128, 0, st>>>(L, reinterpret_cast<const double2*>(alm), nf, noise, out);
    return cudaGetLastError();
}

cudaError_t launch_cl_backward(int L, const double* alm, int nf, const double* gcl, double* galm, double* gnoise,
                               cudaStream_t st) {
    dim3 grid((L + 1 + 127) / 128, L + 1, nf);
    cl_backward_kernel<<<grid, 128, 0, st>>>(L, reinterpret_cast<const double2*>(alm), nf, gcl,
                                             reinterpret_cast<double2*>(galm));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !gnoise) return e;
    noise_grad_kernel<<<(nf * nf + 127) / 128, 128, 0, st>>>(L, nf, gcl, gnoise);
    return cudaGetLastError();
}

cudaError_t launch_bin(int L, const double* cl, int nspec, const int* edges, int nbin, double* out, cudaStream_t st) {
    const int n = nspec * nbin;
    bin_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, cl, nspec, edges, nbin, out);
    return cudaGetLastError();
}

cudaError_t launch_bin_backward(int L, const double* gb, int nspec, const int* edges, int nbin, double* gcl,
                                cudaStream_t st) {
    const int n = nspec * (L + 1);
    bin_backward_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, gb, nspec, edges, nbin, gcl);
    return cudaGetLastError();
}

cudaError_t launch_combine(int L, const double* src, int nsrc, const double* coef, int nout, const double* nsrc_v,
                           double* out, double* nout_v, cudaStream_t st) {
    const int64_t M = (int64_t)(L + 1) * (L + 2) / 2;
    combine_kernel<<<1024, 256, 0, st>>>(M, reinterpret_cast<const double2*>(src), nsrc, coef, nout,
                                         reinterpret_cast<double2*>(out));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !nsrc_v || !nout_v) return e;
    combine_noise_kernel<<<(nout * nout + 127) / 128, 128, 0, st>>>(nsrc_v, nsrc, coef, nout, nout_v);
    return cudaGetLastError();
}

cudaError_t launch_shot_noise(const PrepParams& pp, int is_f64, double* partial, int nblk, double* out,
                              cudaStream_t st) {
    dim3 grid(nblk, pp.ncat);
    if (pp.ncat > 0) {
        if (is_f64) sumsq_kernel<double><<<grid, 256, 0, st>>>(pp, partial, nblk);
        else sumsq_kernel<float><<<grid, 256, 0, st>>>(pp, partial, nblk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    noise_final_kernel<<<(pp.nfield * pp.nfield + 63) / 64, 64, 0, st>>>(pp, partial, nblk, out);
    return cudaGetLastError();
}

}  // namespace psht
