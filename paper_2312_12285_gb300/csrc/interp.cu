// interp.cu -- the paper's interpolated transform (App. "Interpolation") on
// the GPU: y_lm is sampled (value and theta-derivative) on N points
// equispaced in theta, s_k = (k + 1/2) h, h = pi/N, each catalog point
// interpolates it by the cubic Hermite spline of its interval, and the sum
// over points is taken first, per order m:
//
//   v^(m)_{j alpha} = sum_{r in interval j} w_r e^{-i m phi_r} c_alpha(t_r)      (binning)
//   Vy_k = v_{k,0} + v_{k-1,2},  Vd_k = v_{k,1} + v_{k-1,3}                  (fold)
//   a_lm = sum_k [Vy_k y_lm(s_k) + h Vd_k dy_lm/dtheta(s_k)]                 (grid transform)
//
// The intervals j = -1 and N-1 reach ghost samples at -h/2 and pi + h/2,
// continued across the poles as y(-theta) = (-1)^m y(theta) and
// y'(-theta) = (-1)^(m+1) y'(theta); they fold onto samples 0 and N-1.
//
// The theta-derivative is taken in its order-coupled form,
//   dlambda_lm/dtheta = 1/2 [sqrt((l-m)(l+m+1)) lambda_{l,m+1} - sqrt((l+m)(l-m+1)) lambda_{l,m-1}],
//   lambda_{l,-1} = -lambda_{l,1},
// equal to App. A's (l x lambda_l - ... lambda_{l-1}) / sin theta but free of
// its cancellation near the poles (which multiplies the FP32 recurrence's
// error there by ~1/theta) and of the 1/sin weights.  So the derivative
// weights of order m enter the transforms of orders m +- 1: the transform at
// order m carries three weight columns per sample,
//   C0 = Vy^(m),  C1 = h Vd^(m-1),  C2 = h Vd^(m+1),
// run by the mixed tensor-core kernel in its table mode (mixed.cu), and
//   a_lm = T_{l,m} + 1/2 sqrt((l-m)(l+m+1)) U+_{l,m+1} - 1/2 sqrt((l+m)(l-m+1)) U-_{l,m-1}
// (m = 0: T_{l,0} + sqrt(l(l+1)) U+_{l,1}) is combined in FP64 here, with
// T, U+, U- the transforms of C0, C1, C2.
//
// A south sample s_{N-1-k} = pi - s_k has |x| and sin of s_k, and
// lambda_lm(-x) = (-1)^(l+m) lambda_lm(x): both share one position of the
// transform (north weights in columns 0..2, south in 3..5), and the parity
// is applied in the combination.  Positions carry u = x - 1 = -2 sin^2(s/2),
// exact to FP32 relative precision next to the pole.
//
// Kernels: ip_prep (per-point interval, spline weights, turn), ip_hist /
// ip_scan_* / ip_scatter (stable counting sort of the points by interval,
// deterministic), ip_bin (binning, one warp per
// (interval, block of 256 orders), lanes over m, phases by exact fixed-point
// turns and a 32-step rotation), ip_fold (sample weights Vy, Vd in |x|
// order, column maxima), ip_nodes (sample geometry) and ip_combine.
#include "common.cuh"

namespace psht {

constexpr int IP_RANGE = 65536;  // points per range of the counting sort
constexpr int IP_MCHUNK = 256;   // orders per binning task (8 per lane)

// interval j (-1..N-1) and parameter t of cos(theta) = x; +1 gives the bucket
__device__ __forceinline__ int ip_interval(float x, int ntheta, double& t) {
    double xd = (double)x;
    xd = xd > 1.0 ? 1.0 : (xd < -1.0 ? -1.0 : xd);
    const double h = 3.14159265358979323846 / (double)ntheta;
    const double u = acos(xd) / h - 0.5;
    int j = (int)floor(u);
    j = j < -1 ? -1 : (j > ntheta - 1 ? ntheta - 1 : j);
    double tt = u - (double)j;
    t = tt < 0.0 ? 0.0 : (tt > 1.0 ? 1.0 : tt);
    return j;
}

__device__ __forceinline__ bool ip_range_of(const InterpParams& p, int64_t r, int& c, int64_t& i0, int64_t& i1) {
    c = 0;
    while (c + 1 < p.ncat && p.range0[c + 1] <= r) ++c;
    i0 = (r - p.range0[c]) * IP_RANGE;
    i1 = min(p.cat[c].n, i0 + IP_RANGE);
    return i0 < i1;
}

// ------------------------------------------------------ counting sort --
// Per point, in the field's catalog order (index = range * IP_RANGE + offset,
// ranges numbered across catalogs): bucket (interval + 1), w coeff c_alpha(t)
// and the phi turn.  All FP64 arithmetic of the preparation happens here, in
// a fully parallel grid; the sort kernels below only count and move words.
__global__ void __launch_bounds__(256) ip_prep_kernel(const __grid_constant__ InterpParams p) {
    const int64_t nslot = p.nranges * IP_RANGE;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nslot; e += (int64_t)gridDim.x * blockDim.x) {
        int c;
        int64_t i0, i1;
        const int64_t r = e / IP_RANGE;
        if (!ip_range_of(p, r, c, i0, i1)) continue;
        const int64_t i = i0 + (e - r * IP_RANGE);
        if (i >= i1) continue;
        const InterpCat& cd = p.cat[c];
        const float x = cd.x[i], ph = cd.phi[i], w = cd.w[i];
        const bool ok = isfinite(x) && isfinite(ph) && isfinite(w) && fabsf(x) <= 1.f;
        if (!ok) atomicOr(p.err, ERR_RANGE);
        double t;
        const int b = ip_interval(ok ? x : 0.f, p.ntheta, t) + 1;
        const double wv = ok ? cd.coeff * (double)w : 0.0;
        const double v = 1.0 - t;
        const uint64_t turn = phi_to_turn(ok ? (double)ph : 0.0);
        const int64_t S = p.nranges * IP_RANGE;
        p.stage[e] = (uint32_t)b;
        p.stage[S + e] = __float_as_uint((float)(wv * (2.0 * t + 1.0) * v * v));
        p.stage[2 * S + e] = __float_as_uint((float)(wv * t * v * v));
        p.stage[3 * S + e] = __float_as_uint((float)(wv * t * t * (3.0 - 2.0 * t)));
        p.stage[4 * S + e] = __float_as_uint((float)(wv * t * t * (t - 1.0)));
        p.stage[5 * S + e] = (uint32_t)(turn >> 32);
        p.stage[6 * S + e] = (uint32_t)(turn & 0xffffffffu);
    }
}

__global__ void __launch_bounds__(256) ip_hist_kernel(const __grid_constant__ InterpParams p) {
    extern __shared__ int cnt[];
    const int64_t r = blockIdx.x;
    for (int b = threadIdx.x; b < p.nb; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    int c;
    int64_t i0, i1;
    if (ip_range_of(p, r, c, i0, i1)) {
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
            atomicAdd(&cnt[p.stage[r * IP_RANGE + (i - i0)]], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < p.nb; b += blockDim.x) p.hist[r * p.nb + b] = cnt[b];
}

// per bucket: prefix over ranges (in place) and the bucket total
__global__ void ip_scan_ranges_kernel(const __grid_constant__ InterpParams p) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.nb) return;
    int64_t run = 0;
    for (int64_t r = 0; r < p.nranges; ++r) {
        const int h = p.hist[r * p.nb + b];
        p.hist[r * p.nb + b] = (int32_t)run;
        run += h;
    }
    p.total[b] = run;
}

// exclusive scan of the bucket totals (one CTA)
__global__ void __launch_bounds__(1024) ip_scan_buckets_kernel(const __grid_constant__ InterpParams p) {
    __shared__ int64_t part[1024];
    const int per = (p.nb + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    int64_t s = 0;
    for (int b = b0; b < min(p.nb, b0 + per); ++b) s += p.total[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int k = 0; k < 1024; ++k) {
            const int64_t v = part[k];
            part[k] = run;
            run += v;
        }
        p.binoff[p.nb] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int b = b0; b < min(p.nb, b0 + per); ++b) {
        p.binoff[b] = run;
        run += p.total[b];
    }
}

// stable scatter: one warp per range, points in index order, four 32-point
// chunks per iteration so that their loads are in flight together
__global__ void __launch_bounds__(32) ip_scatter_kernel(const __grid_constant__ InterpParams p) {
    extern __shared__ int32_t next[];  // point counts of one field stay below 2^31 (checked on the host)
    const int64_t r = blockIdx.x;
    const int lane = threadIdx.x;
    for (int b = lane; b < p.nb; b += 32) next[b] = (int32_t)(p.binoff[b] + p.hist[r * p.nb + b]);
    __syncwarp();
    int c;
    int64_t i0, i1;
    if (!ip_range_of(p, r, c, i0, i1)) return;
    const int64_t S = p.nranges * IP_RANGE;
    const int64_t e0 = r * IP_RANGE - i0;  // stage slot of point i is e0 + i
    constexpr int U = 4;
    for (int64_t base = i0; base < i1; base += 32 * U) {
        uint32_t v[U][7];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + 32 * u + lane;
#pragma unroll
            for (int a = 0; a < 7; ++a) v[u][a] = i < i1 ? p.stage[a * S + e0 + i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = base + 32 * u + lane;
            const bool valid = i < i1;
            const int b = valid ? (int)v[u][0] : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, b);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            int64_t dst = 0;
            if (valid) dst = next[b] + rank;
            __syncwarp();
            if (valid && rank == 0) next[b] += __popc(peers);
            __syncwarp();
            if (valid) {
                reinterpret_cast<uint32_t*>(p.wc)[dst] = v[u][1];
                reinterpret_cast<uint32_t*>(p.wc)[p.npts + dst] = v[u][2];
                reinterpret_cast<uint32_t*>(p.wc)[2 * p.npts + dst] = v[u][3];
                reinterpret_cast<uint32_t*>(p.wc)[3 * p.npts + dst] = v[u][4];
                p.turn[dst] = v[u][5];
                p.turn[p.npts + dst] = v[u][6];
            }
        }
    }
}

// -------------------------------------------------------------- binning --
__device__ __forceinline__ float2 mx_fma2_ip(float2 a, float2 b, float2 c) {
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(reinterpret_cast<unsigned long long&>(d))
        : "l"(reinterpret_cast<unsigned long long&>(a)), "l"(reinterpret_cast<unsigned long long&>(b)),
          "l"(reinterpret_cast<unsigned long long&>(c)));
    return d;
}

// v^(m)_{j alpha} for one interval and 256 orders per warp: lane l holds
// m = 256 c + l + 32 k, k = 0..7, as (re, im) of the 4 alpha.  The interval's
// points are read in batches of 32, one point per lane (coalesced), the next
// batch while the current one runs; the lane that read a point also computes
// its 32-order phase step, and each point's words reach every lane by
// shuffles.
__global__ void __launch_bounds__(256) ip_bin_kernel(const __grid_constant__ InterpParams p) {
    const int lane = threadIdx.x & 31;
    const int nch = (p.lmax + IP_MCHUNK) / IP_MCHUNK;
    const int64_t ntask = (int64_t)p.nb * nch;
    const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < ntask; task += nwarp) {
        const int b = (int)(task / nch), c = (int)(task - (int64_t)(task / nch) * nch);
        const int m0 = IP_MCHUNK * c + lane;
        // per m: (re, im) of the alpha pairs {0, 1} and {2, 3} as f32x2 lanes
        float2 vr01[8], vi01[8], vr23[8], vi23[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) vr01[k] = vi01[k] = vr23[k] = vi23[k] = make_float2(0.f, 0.f);
        const int64_t r0 = p.binoff[b], r1 = p.binoff[b + 1];
        // orders of this block that exist (the last block of the range may be partial)
        const int kmax = min(8, (p.lmax - IP_MCHUNK * c) / 32 + 1);
        // this lane's point of the next batch
        float n0 = 0.f, n1 = 0.f, n2 = 0.f, n3 = 0.f;
        uint32_t nth = 0u, ntl = 0u;
        auto load = [&](int64_t r) {
            if (r < r1) {
                n0 = p.wc[r];
                n1 = p.wc[p.npts + r];
                n2 = p.wc[2 * p.npts + r];
                n3 = p.wc[3 * p.npts + r];
                nth = p.turn[r];
                ntl = p.turn[p.npts + r];
            }
        };
        load(r0 + lane);
        for (int64_t rb = r0; rb < r1; rb += 32) {
            const float q0 = n0, q1 = n1, q2 = n2, q3 = n3;
            const uint32_t qth = nth, qtl = ntl;
            float qc32, qs32;  // e^{-32 i phi} of this lane's point
            phase_f32(32, qth, qtl, qc32, qs32);
            load(rb + 32 + lane);
            const int cnt = (int)min((int64_t)32, r1 - rb);
            for (int j = 0; j < cnt; ++j) {
                const float2 w01 = make_float2(__shfl_sync(0xffffffffu, q0, j), __shfl_sync(0xffffffffu, q1, j));
                const float2 w23 = make_float2(__shfl_sync(0xffffffffu, q2, j), __shfl_sync(0xffffffffu, q3, j));
                const uint32_t th = __shfl_sync(0xffffffffu, qth, j), tl = __shfl_sync(0xffffffffu, qtl, j);
                const float2 nw01 = make_float2(-w01.x, -w01.y), nw23 = make_float2(-w23.x, -w23.y);
                const float c32 = __shfl_sync(0xffffffffu, qc32, j), s32 = __shfl_sync(0xffffffffu, qs32, j);
                float cs, sn;
                phase_f32(m0, th, tl, cs, sn);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (k >= kmax) break;
                    // w c_alpha e^{-i m phi} = w c_alpha (cos - i sin)
                    const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn);
                    vr01[k] = mx_fma2_ip(w01, c2, vr01[k]);
                    vi01[k] = mx_fma2_ip(nw01, s2, vi01[k]);
                    vr23[k] = mx_fma2_ip(w23, c2, vr23[k]);
                    vi23[k] = mx_fma2_ip(nw23, s2, vi23[k]);
                    const float cn = fmaf(cs, c32, -sn * s32);
                    sn = fmaf(sn, c32, cs * s32);
                    cs = cn;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int m = m0 + 32 * k;
            if (m <= p.lmax) {
                float4* dst = reinterpret_cast<float4*>(p.v + ((int64_t)m * p.nb + b) * 4);
                dst[0] = make_float4(vr01[k].x, vi01[k].x, vr01[k].y, vi01[k].y);
                dst[1] = make_float4(vr23[k].x, vi23[k].x, vr23[k].y, vi23[k].y);
            }
        }
    }
}

// sample weights (Vy, Vd) of every order at each sample's position (north
// and mirrored south halves); column maxima max|Vy| and h max|Vd|
__global__ void __launch_bounds__(256) ip_fold_kernel(const __grid_constant__ InterpParams p) {
    const int N = p.ntheta;
    const int64_t total = (int64_t)(p.lmax + 1) * N;
    const float h = (float)(3.14159265358979323846 / (double)N);
    unsigned my = 0u, md = 0u;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / N), k = (int)(e - (int64_t)m * N);
        const float2* vm = p.v + (int64_t)m * p.nb * 4;
        // interval k (bucket k + 1): sample k is its left end; interval k - 1
        // (bucket k): its right end
        const float2 a0 = vm[(k + 1) * 4 + 0], a1 = vm[(k + 1) * 4 + 1];
        const float2 b2 = vm[k * 4 + 2], b3 = vm[k * 4 + 3];
        float2 vy = make_float2(a0.x + b2.x, a0.y + b2.y);
        float2 vd = make_float2(a1.x + b3.x, a1.y + b3.y);
        const float sg = (m & 1) ? -1.f : 1.f;
        if (k == 0) {  // ghost at -h/2 = left end of interval -1 (bucket 0)
            const float2 g0 = vm[0], g1 = vm[1];
            vy.x += sg * g0.x;
            vy.y += sg * g0.y;
            vd.x -= sg * g1.x;
            vd.y -= sg * g1.y;
        }
        if (k == N - 1) {  // ghost at pi + h/2 = right end of interval N-1 (bucket N)
            const float2 g2 = vm[N * 4 + 2], g3 = vm[N * 4 + 3];
            vy.x += sg * g2.x;
            vy.y += sg * g2.y;
            vd.x -= sg * g3.x;
            vd.y -= sg * g3.y;
        }
        // north sample k at position k, south sample N-1-k at the same position
        const int half = k >= N / 2;
        const int64_t pos = half ? N - 1 - k : k;
        float4* dst = reinterpret_cast<float4*>(p.vtab + ((int64_t)m * p.ntot + pos) * 4 + 2 * half);
        *dst = make_float4(vy.x, vy.y, vd.x, vd.y);
        my = max(my, __float_as_uint(fmaxf(fabsf(vy.x), fabsf(vy.y))));
        md = max(md, __float_as_uint(h * fmaxf(fabsf(vd.x), fabsf(vd.y))));
    }
    my = __reduce_max_sync(0xffffffffu, my);
    md = __reduce_max_sync(0xffffffffu, md);
    if ((threadIdx.x & 31) == 0) {
        if (my) {
            atomicMax(&p.colmax[0], my);
            atomicMax(&p.colmax[3], my);
        }
        if (md) {
            atomicMax(&p.colmax[1], md);
            atomicMax(&p.colmax[2], md);
            atomicMax(&p.colmax[4], md);
            atomicMax(&p.colmax[5], md);
        }
    }
}

// zero weights of the padding positions N..ntot-1 of every order
__global__ void ip_pad_kernel(const __grid_constant__ InterpParams p) {
    const int64_t half = p.ntheta / 2, npad = p.ntot - half;
    const int64_t total = (int64_t)(p.lmax + 1) * npad * 4;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / (npad * 4), rem = e - m * npad * 4;
        p.vtab[(m * p.ntot + half) * 4 + rem] = make_float2(0.f, 0.f);
    }
}

// geometry of the positions in the layout of the mixed kernel: u = x - 1 of
// the north sample (= -2 sin^2(s/2)), log2 sin hi/lo, turn 0; padding at x = 0
__global__ void ip_nodes_kernel(const __grid_constant__ InterpParams p) {
    const int N = p.ntheta;
    const double h = 3.14159265358979323846 / (double)N;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p.ntot; q += (int64_t)gridDim.x * blockDim.x) {
        float x = -1.f, lh = 0.f, ll = 0.f;
        if (q < N / 2) {
            const double th = (q + 0.5) * h;
            const double sh = sin(0.5 * th);
            const double ls = log2(sin(th));
            x = (float)(-2.0 * sh * sh);
            lh = (float)ls;
            ll = (float)(ls - (double)lh);
        }
        float* b = reinterpret_cast<float*>(p.nodes);
        b[q] = x;
        b[p.ntot + q] = lh;
        b[2 * p.ntot + q] = ll;
        p.nodes[3 * p.ntot + q] = 0u;
        p.nodes[4 * p.ntot + q] = 0u;
    }
}

// a_lm = T_lm + 1/2 sqrt((l-m)(l+m+1)) U+_{l,m+1} - 1/2 sqrt((l+m)(l-m+1)) U-_{l,m-1}
// (m = 0: T_l0 + sqrt(l(l+1)) U+_{l,1});  T, U+, U- = transforms of columns 0, 1, 2
// (north) and 3, 4, 5 (south)
__global__ void ip_combine_kernel(int lmax, int64_t nmodes, const double2* T, double2* out) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nmodes;
         idx += (int64_t)gridDim.x * blockDim.x) {
        // (l, m) of the packed m-major index m(2L+1-m)/2 + l; column m starts
        // at start(m) = m(2L+3-m)/2
        int m = (int)((2.0 * lmax + 3.0 - sqrt((2.0 * lmax + 3.0) * (2.0 * lmax + 3.0) - 8.0 * (double)idx)) * 0.5);
        m = m < 0 ? 0 : (m > lmax ? lmax : m);
        while (m > 0 && (int64_t)m * (2 * lmax + 3 - m) / 2 > idx) --m;
        while (m < lmax && (int64_t)(m + 1) * (2 * lmax + 3 - (m + 1)) / 2 <= idx) ++m;
        const int l = (int)(idx - (int64_t)m * (2 * lmax + 1 - m) / 2);
        // transform f at (l, mm): north part + (-1)^(l+mm) south part
        auto X = [&](int f, int mm, int64_t j) {
            const double2 a = T[f * nmodes + j], b = T[(f + 3) * nmodes + j];
            const double sg = ((l + mm) & 1) ? -1.0 : 1.0;
            return make_double2(a.x + sg * b.x, a.y + sg * b.y);
        };
        const double2 t = X(0, m, idx);
        double re = t.x, im = t.y;
        if (l > m) {  // U+ at (l, m + 1)
            const int64_t j = (int64_t)(m + 1) * (2 * lmax - m) / 2 + l;
            const double2 u = X(1, m + 1, j);
            const double c = (m == 0 ? 1.0 : 0.5) * sqrt((double)(l - m) * (double)(l + m + 1));
            re += c * u.x;
            im += c * u.y;
        }
        if (m > 0) {  // U- at (l, m - 1)
            const int64_t j = (int64_t)(m - 1) * (2 * lmax + 2 - m) / 2 + l;
            const double2 u = X(2, m - 1, j);
            const double c = 0.5 * sqrt((double)(l + m) * (double)(l - m + 1));
            re -= c * u.x;
            im -= c * u.y;
        }
        out[idx] = make_double2(re, im);
    }
}

// ------------------------------------------------------------ launchers --
int64_t interp_nranges(int64_t n) { return (n + IP_RANGE - 1) / IP_RANGE; }
int64_t interp_range() { return IP_RANGE; }

cudaError_t launch_interp_sort(const InterpParams& p, cudaStream_t st) {
    if (p.nranges == 0) {
        // no points: empty intervals
        return cudaMemsetAsync(p.binoff, 0, (size_t)(p.nb + 1) * sizeof(int64_t), st);
    }
    const int64_t pblocks = (p.nranges * IP_RANGE + 255) / 256;
    ip_prep_kernel<<<(unsigned)(pblocks < 4096 ? pblocks : 4096), 256, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t hs = (size_t)p.nb * sizeof(int);
    int occ = 0;
    e = configure_kernel(reinterpret_cast<const void*>(ip_hist_kernel), 256, hs, &occ);
    if (e != cudaSuccess) return e;
    ip_hist_kernel<<<(unsigned)p.nranges, 256, hs, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ip_scan_ranges_kernel<<<(p.nb + 255) / 256, 256, 0, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ip_scan_buckets_kernel<<<1, 1024, 0, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t ss = (size_t)p.nb * sizeof(int32_t);
    e = configure_kernel(reinterpret_cast<const void*>(ip_scatter_kernel), 32, ss, &occ);
    if (e != cudaSuccess) return e;
    ip_scatter_kernel<<<(unsigned)p.nranges, 32, ss, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_interp_tables(const InterpParams& p, int sm_count, cudaStream_t st) {
    ip_bin_kernel<<<sm_count * 8, 256, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ip_fold_kernel<<<sm_count * 8, 256, 0, st>>>(p);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (p.ntot > p.ntheta / 2) {
        ip_pad_kernel<<<sm_count * 4, 256, 0, st>>>(p);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ip_nodes_kernel<<<(unsigned)((p.ntot + 255) / 256), 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_interp_combine(int lmax, int64_t nmodes, const double* T, double* out, cudaStream_t st) {
    ip_combine_kernel<<<512, 256, 0, st>>>(lmax, nmodes, reinterpret_cast<const double2*>(T),
                                           reinterpret_cast<double2*>(out));
    return cudaGetLastError();
}

}  // namespace psht
