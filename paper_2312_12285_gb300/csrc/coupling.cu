// coupling.cu -- mode-coupling matrix of the masked pseudo-spectrum (Eq. chat),
// its binned form, the mode decoupling (Eq. mode_coupling, Eq.
// expectation_value) and the FKP-like normalisation (Sec. 2.1).
//
//   M_ll' = (2l'+1)/(4 pi) sum_lambda (2 lambda + 1) (l l' lambda; 0 0 0)^2 W_lambda
//
// The squared 3j symbol with zero orders has the product form
//   (l1 l2 l3; 0 0 0)^2 = b(g-l1) b(g-l2) b(g-l3) / ((2g+1) b(g)),  2g = l1+l2+l3,
//   b(j) = C(2j, j) / 4^j = prod_{k=1..j} (2k-1)/(2k),
// (the closed form of App. "Wigner 3j symbols" squared, the powers of 4
// cancelling), so no recurrence error builds up along lambda and every term
// is three table reads and two FP64 operations.  Writing lambda = 2g - s with
// s = l + l', the factor b(s-g) (2 lambda+1) W_lambda / ((2g+1) b(g) 4 pi)
// depends on (s, g) only: a CTA owns one anti-diagonal s (a slice of its
// pairs l <= l' = s - l), builds that factor T_s[g] in shared memory once, and
// each thread sums
//   K_ll' = sum_{g = l'}^{min(s, (s + lmax_w)/2)} b(g-l) b(g-l') T_s[g]
// (g >= l' is lambda >= |l - l'|; g <= s is lambda <= l + l').  Then
// M_ll' = (2l'+1) K_ll' and M_l'l = (2l+1) K_ll' (K is symmetric).  A warp's
// lanes take consecutive l, so the b reads are consecutive words and T_s[g]
// is a broadcast; lanes whose range starts later read zeros below b(0).
// The FP64 pipe bounds the kernel: ~L^3/6 terms for lmax_w = L.
#include "common.cuh"

#include <math_constants.h>

#include <algorithm>

namespace psht {

constexpr int CP_THREADS = 256;
constexpr int CP_PAD = 32;  // zeros below b(0) in shared memory

// b(j) for 0 <= j < n and ib(g) = 1 / ((2g+1) b(g)): one thread, sequential
// product (deterministic; ~n ulp at most).
__global__ void cp_tables_kernel(int n, double* __restrict__ b, double* __restrict__ ib) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double v = 1.0;
    for (int j = 0; j < n; ++j) {
        if (j > 0) v *= (double)(2 * j - 1) / (double)(2 * j);
        b[j] = v;
        ib[j] = 1.0 / ((double)(2 * j + 1) * v);
    }
}

__global__ void __launch_bounds__(CP_THREADS) cp_coupling_kernel(int L, int Lw, const double* __restrict__ W,
                                                                 const double* __restrict__ b,
                                                                 const double* __restrict__ ib,
                                                                 double* __restrict__ M) {
    extern __shared__ double cp_smem[];
    const int s = blockIdx.y;
    const int llo = max(0, s - L), lhi = s >> 1;
    const int first = llo + blockIdx.x * CP_THREADS;
    if (first > lhi) return;
    const int g0 = (s + 1) >> 1;
    const int g1 = min(s, (s + Lw) >> 1);
    double* bs = cp_smem + CP_PAD;    // b(-CP_PAD .. s)
    double* Ts = bs + s + 1;          // T_s[g - g0], g0 <= g <= g1
    for (int j = threadIdx.x - CP_PAD; j <= s; j += CP_THREADS) bs[j] = j < 0 ? 0.0 : b[j];
    __syncthreads();
    const double inv4pi = 1.0 / (4.0 * CUDART_PI);
    for (int g = g0 + threadIdx.x; g <= g1; g += CP_THREADS) {
        const int lam = 2 * g - s;
        Ts[g - g0] = bs[s - g] * ib[g] * ((double)(2 * lam + 1) * W[lam] * inv4pi);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wfirst = first + warp * 32;
    if (wfirst > lhi) return;
    const int wlast = min(wfirst + 31, lhi);
    const int lraw = wfirst + lane;
    const int l = min(lraw, wlast);  // lanes past the last pair repeat it and store nothing
    const int lp = s - l;
    // g from the warp's smallest start s - wlast; a lane with l < wlast starts
    // contributing at g = lp (below it b(g - lp) reads the zero padding).
    const double* bl = bs - l;    // bl[g] = b(g - l)
    const double* blp = bs - lp;  // blp[g] = b(g - l'), zero for g < l'
    const double* T = Ts - g0;
    // four independent accumulators (FP64 latency), combined in a fixed tree
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    int g = s - wlast;
    for (; g + 3 <= g1; g += 4) {
        acc0 = fma(bl[g] * blp[g], T[g], acc0);
        acc1 = fma(bl[g + 1] * blp[g + 1], T[g + 1], acc1);
        acc2 = fma(bl[g + 2] * blp[g + 2], T[g + 2], acc2);
        acc3 = fma(bl[g + 3] * blp[g + 3], T[g + 3], acc3);
    }
    for (; g <= g1; ++g) acc0 = fma(bl[g] * blp[g], T[g], acc0);
    if (lraw <= wlast) {
        const double K = (acc0 + acc1) + (acc2 + acc3);
        M[(int64_t)l * (L + 1) + lp] = (double)(2 * lp + 1) * K;
        if (lp != l) M[(int64_t)lp * (L + 1) + l] = (double)(2 * l + 1) * K;
    }
}

size_t coupling_smem_bytes(int L) { return (size_t)(CP_PAD + 2 * L + 1 + L + 2) * sizeof(double); }

cudaError_t launch_coupling(int L, int Lw, const double* W, double* M, double* b, double* ib, cudaStream_t st) {
    const int n = 2 * L + 1;
    cp_tables_kernel<<<1, 1, 0, st>>>(n, b, ib);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = coupling_smem_bytes(L);
    int occ = 0;
    if ((e = configure_kernel((const void*)cp_coupling_kernel, CP_THREADS, smem, &occ)) != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int npair_max = L / 2 + 1;
    dim3 grid((npair_max + CP_THREADS - 1) / CP_THREADS, 2 * L + 1);
    cp_coupling_kernel<<<grid, CP_THREADS, smem, st>>>(L, Lw, W, b, ib, M);
    return cudaGetLastError();
}

// ------------------------------------------------------------ binning --
// Bin edges are clamped into [0, L+1] and made non-decreasing on the device,
// so a malformed edge array cannot send a read outside M.
__device__ __forceinline__ void cp_edges(const int* __restrict__ edges, int b, int L, int& lo, int& hi) {
    lo = min(max(edges[b], 0), L + 1);
    hi = min(max(edges[b + 1], lo), L + 1);
}

// R[b][l'] = sum_{l in b} M[l][l'] / Delta_b (theta_b^l = 1/Delta_l, Sec. 2.1)
__global__ void cp_bin_rows_kernel(int L, const double* __restrict__ M, const int* __restrict__ edges, int nbin,
                                   double* __restrict__ R) {
    const int b = blockIdx.y;
    const int lp = blockIdx.x * blockDim.x + threadIdx.x;
    if (lp > L) return;
    int lo, hi;
    cp_edges(edges, b, L, lo, hi);
    double acc = 0.0;
    for (int l = lo; l < hi; ++l) acc += M[(int64_t)l * (L + 1) + lp];
    R[(int64_t)b * (L + 1) + lp] = hi > lo ? acc / (double)(hi - lo) : 0.0;
}

// Mbb[b][b'] = sum_{l' in b'} R[b][l']: one warp per entry, fixed-order
// lane-strided sums and a fixed shuffle tree.
__global__ void cp_bin_cols_kernel(int L, const double* __restrict__ R, const int* __restrict__ edges, int nbin,
                                   double* __restrict__ Mbb) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nbin * nbin) return;
    const int b = gw / nbin, b2 = gw % nbin;
    int lo, hi;
    cp_edges(edges, b2, L, lo, hi);
    double acc = 0.0;
    for (int lp = lo + lane; lp < hi; lp += 32) acc += R[(int64_t)b * (L + 1) + lp];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Mbb[(int64_t)b * nbin + b2] = acc;
}

cudaError_t launch_coupling_binned(int L, const double* M, const int* edges, int nbin, double* R, double* Mbb,
                                   cudaStream_t st) {
    dim3 g1((L + 1 + 255) / 256, nbin);
    cp_bin_rows_kernel<<<g1, 256, 0, st>>>(L, M, edges, nbin, R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t threads = (int64_t)nbin * nbin * 32;
    cp_bin_cols_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(L, R, edges, nbin, Mbb);
    return cudaGetLastError();
}

// ---------------------------------------------------------- decoupling --
// Gauss-Jordan inverse of the n x n binned coupling with partial pivoting
// (largest |pivot|, lowest row on ties), one CTA, augmented matrix [A | I]
// in the workspace.  A zero or non-finite pivot marks the matrix singular:
// the inverse is then written as NaN.
constexpr int CP_INV_THREADS = 1024;

__global__ void __launch_bounds__(CP_INV_THREADS) cp_invert_kernel(int n, const double* __restrict__ A,
                                                                   double* __restrict__ aug,
                                                                   double* __restrict__ Ainv) {
    __shared__ double rv[CP_INV_THREADS / 32];
    __shared__ int ri[CP_INV_THREADS / 32];
    __shared__ int piv;
    __shared__ int singular;
    extern __shared__ double fac[];  // [n] column factors of the current step
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int w2 = 2 * n;
    for (int e = t; e < n * w2; e += blockDim.x) {
        const int r = e / w2, c = e % w2;
        aug[e] = c < n ? A[(int64_t)r * n + c] : (c - n == r ? 1.0 : 0.0);
    }
    if (t == 0) singular = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // pivot: argmax_{r >= k} |aug[r][k]|, lowest r on ties
        double best = -1.0;
        int bi = n;
        for (int r = k + t; r < n; r += blockDim.x) {
            const double v = fabs(aug[(int64_t)r * w2 + k]);
            if (v > best) {
                best = v;
                bi = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            rv[warp] = best;
            ri[warp] = bi;
        }
        __syncthreads();
        if (t == 0) {
            double bv = rv[0];
            int bidx = ri[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (rv[w] > bv || (rv[w] == bv && ri[w] < bidx)) {
                    bv = rv[w];
                    bidx = ri[w];
                }
            piv = bidx;
            if (!(bv > 0.0) || !isfinite(bv) || bidx >= n) singular = 1;
        }
        __syncthreads();
        if (singular) break;
        const int p = piv;
        if (p != k)
            for (int c = t; c < w2; c += blockDim.x) {
                const double a = aug[(int64_t)k * w2 + c];
                aug[(int64_t)k * w2 + c] = aug[(int64_t)p * w2 + c];
                aug[(int64_t)p * w2 + c] = a;
            }
        __syncthreads();
        const double inv = 1.0 / aug[(int64_t)k * w2 + k];
        __syncthreads();
        for (int c = t; c < w2; c += blockDim.x) aug[(int64_t)k * w2 + c] *= inv;
        for (int r = t; r < n; r += blockDim.x) fac[r] = r == k ? 0.0 : aug[(int64_t)r * w2 + k];
        __syncthreads();
        for (int e = t; e < n * w2; e += blockDim.x) {
            const int r = e / w2, c = e % w2;
            if (r != k) aug[e] = fma(-fac[r], aug[(int64_t)k * w2 + c], aug[e]);
        }
        __syncthreads();
    }
    for (int e = t; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e % n;
        Ainv[e] = singular ? CUDART_NAN : aug[(int64_t)r * w2 + n + c];
    }
}

// Mcal[b][l'] = sum_b' Minv[b][b'] R[b'][l']   (Eq. expectation_value)
__global__ void cp_apply_rows_kernel(int L, int nbin, const double* __restrict__ Minv, const double* __restrict__ R,
                                     double* __restrict__ Mcal) {
    const int b = blockIdx.y;
    const int lp = blockIdx.x * blockDim.x + threadIdx.x;
    if (lp > L) return;
    double acc = 0.0;
    for (int b2 = 0; b2 < nbin; ++b2) acc = fma(Minv[(int64_t)b * nbin + b2], R[(int64_t)b2 * (L + 1) + lp], acc);
    Mcal[(int64_t)b * (L + 1) + lp] = acc;
}

// out[s][b] = sum_b' Minv[b][b'] cl[s][b']   (Eq. mode_coupling)
__global__ void cp_apply_spectra_kernel(int nbin, int nspec, const double* __restrict__ Minv,
                                        const double* __restrict__ cl, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nspec * nbin) return;
    const int s = t / nbin, b = t % nbin;
    double acc = 0.0;
    for (int b2 = 0; b2 < nbin; ++b2) acc = fma(Minv[(int64_t)b * nbin + b2], cl[(int64_t)s * nbin + b2], acc);
    out[t] = acc;
}

size_t decouple_workspace_bytes(int nbin) { return (size_t)nbin * 2 * nbin * sizeof(double); }

cudaError_t launch_decouple(int L, int nbin, const double* Mbb, const double* R, const double* cl, int nspec,
                            double* Minv, double* Mcal, double* cl_dec, double* aug, cudaStream_t st) {
    cp_invert_kernel<<<1, CP_INV_THREADS, (size_t)nbin * sizeof(double), st>>>(nbin, Mbb, aug, Minv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (R && Mcal) {
        dim3 g((L + 1 + 255) / 256, nbin);
        cp_apply_rows_kernel<<<g, 256, 0, st>>>(L, nbin, Minv, R, Mcal);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (cl && cl_dec && nspec > 0) {
        cp_apply_spectra_kernel<<<(nspec * nbin + 127) / 128, 128, 0, st>>>(nbin, nspec, Minv, cl, cl_dec);
        e = cudaGetLastError();
    }
    return e;
}

// ------------------------------------------------------ normalisation --
// norm = 1 / [sum_l (2l+1) W_l / 4 pi]: one CTA, fixed-order strided sums and
// a fixed shared-memory tree.
__global__ void __launch_bounds__(256) cp_fkp_norm_kernel(int Lw, const double* __restrict__ W,
                                                          double* __restrict__ norm) {
    __shared__ double part[256];
    double acc = 0.0;
    for (int l = threadIdx.x; l <= Lw; l += 256) acc = fma((double)(2 * l + 1), W[l], acc);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) norm[0] = 1.0 / (part[0] / (4.0 * CUDART_PI));
}

__global__ void cp_scale_kernel(int64_t n, const double* __restrict__ norm, const double* __restrict__ in,
                                double* __restrict__ out) {
    const double f = norm[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = f * in[i];
}

cudaError_t launch_fkp_normalise(int Lw, const double* W, int L, int nbin, const double* R, const double* cl,
                                 int nspec, double* norm, double* Mprime, double* cl_norm, cudaStream_t st) {
    cp_fkp_norm_kernel<<<1, 256, 0, st>>>(Lw, W, norm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (R && Mprime) {
        const int64_t n = (int64_t)nbin * (L + 1);
        cp_scale_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(n, norm, R, Mprime);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (cl && cl_norm && nspec > 0) {
        const int64_t n = (int64_t)nspec * nbin;
        cp_scale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, norm, cl, cl_norm);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace psht
