// spai.cu -- learned sparse-approximate-inverse right preconditioner:
// features, an 8 -> 64 -> 64 -> 1 MLP per nonzero of A, the probe loss
// L = 1/(2 P n) sum_p ||A M z_p - z_p||^2 with its gradients, Adam, and
// inference of M's values for right-preconditioned GMRES (A M y = b,
// x = M y).  C-ABI gmres_spai_* in include/gmres_gb300.h.
//
// M has A's sparsity pattern and m_pq = g_pq / a_pp, g = MLP(features of
// (p, q)).  Features (per nonzero, d = diagonal, a zero diagonal counts as 1):
//   a_pq/d_p, d_q/d_p, [p==q], sum|a_p.|/|d_p|, sum|a_.q|/|d_q|, nnz(p)/8,
//   sign(a_pq), sign(q-p).
// Everything runs in binary32 on the device; sums over nonzeros go through
// per-block partials reduced by the last block in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/gmres_gb300.h"
#include "grid_kernels.cuh"
#include "handle.hpp"
#include "host_util.hpp"

using namespace gmres;
using namespace gmres_host;

namespace {

constexpr int NF = 8, NH = 64;
constexpr int P_W1 = 0, P_B1 = P_W1 + NH * NF, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH,
              P_W3 = P_B2 + NH, P_B3 = P_W3 + NH, NPARAM = P_B3 + 1;
static_assert(NPARAM == GMRES_SPAI_NPARAM, "parameter count");
constexpr int TK = 64;        // nonzeros per backward tile
constexpr int TKP = TK + 1;   // padded tile row (bank-conflict free)
constexpr int BWD_THREADS = 256;

// Per-row diagonal (1 when missing or zero) and absolute row sum.
__global__ void k_rowstats(int n, const int *rowptr, const int *colind, const double *vals,
                           float *dinv, float *rowabs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 1.0, s = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            s += fabs(vals[k]);
            if (colind[k] == i && vals[k] != 0.0)
                d = vals[k];
        }
        dinv[i] = (float)(1.0 / d);
        rowabs[i] = (float)(s / fabs(d));
    }
}

// Absolute column sums from the CSR of A^T, divided by |d_q|.
__global__ void k_colstats(int n, const int *trowptr, const double *tvals, const float *dinv,
                           float *colabs) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = trowptr[q]; k < trowptr[q + 1]; ++k)
            s += fabs(tvals[k]);
        colabs[q] = (float)(s * fabs((double)dinv[q]));
    }
}

// Features, feature-major: feat[f * nnz + k]; slot 8 holds 1/d_p.
__global__ void k_features(int n, int64_t nnz, const int *rowptr, const int *colind,
                           const double *vals, const float *dinv, const float *rowabs,
                           const float *colabs, float *feat) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const double dp_inv = dinv[p];
        const int beg = rowptr[p], end = rowptr[p + 1];
        for (int k = beg; k < end; ++k) {
            const int q = colind[k];
            const double a = vals[k];
            feat[0 * nnz + k] = (float)(a * dp_inv);
            feat[1 * nnz + k] = (float)(dp_inv / (double)dinv[q]);
            feat[2 * nnz + k] = (p == q) ? 1.f : 0.f;
            feat[3 * nnz + k] = rowabs[p];
            feat[4 * nnz + k] = colabs[q];
            feat[5 * nnz + k] = (float)(end - beg) * 0.125f;
            feat[6 * nnz + k] = (float)((a > 0) - (a < 0));
            feat[7 * nnz + k] = (float)((q > p) - (q < p));
            feat[8 * nnz + k] = (float)dp_inv;
        }
    }
}

// MLP forward per nonzero; m = g / d_p.  H1 / H2 (feature-major, nullable)
// keep the activations for the backward pass.
__global__ void __launch_bounds__(256) k_mlp_fwd(int64_t nnz, const float *feat,
                                                 const float *params, float *m32, double *m64,
                                                 float *H1, float *H2) {
    __shared__ __align__(16) float w[NPARAM + 3];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x)
        w[i] = params[i];
    __syncthreads();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        float f[NF];
#pragma unroll
        for (int j = 0; j < NF; ++j)
            f[j] = feat[j * nnz + k];
        float h1[NH];
#pragma unroll
        for (int o = 0; o < NH; ++o) {
            float a = w[P_B1 + o];
#pragma unroll
            for (int j = 0; j < NF; ++j)
                a += w[P_W1 + o * NF + j] * f[j];
            h1[o] = fmaxf(a, 0.f);
            if (H1)
                H1[o * nnz + k] = h1[o];
        }
        float g = w[P_B3];
#pragma unroll 4
        for (int o = 0; o < NH; ++o) {
            const float4 *row = reinterpret_cast<const float4 *>(w + P_W2 + o * NH);
            float a = w[P_B2 + o];
#pragma unroll
            for (int i4 = 0; i4 < NH / 4; ++i4) {
                float4 q = row[i4];
                a += q.x * h1[4 * i4] + q.y * h1[4 * i4 + 1] + q.z * h1[4 * i4 + 2] +
                     q.w * h1[4 * i4 + 3];
            }
            const float h2 = fmaxf(a, 0.f);
            if (H2)
                H2[o * nnz + k] = h2;
            g += w[P_W3 + o] * h2;
        }
        const float m = g * feat[8 * nnz + k];
        if (m32)
            m32[k] = m;
        if (m64)
            m64[k] = (double)m;
    }
}

// r = A u - z and the partial sums of ||r||^2 (binary64) per block.
__global__ void k_probe_residual(int n, const float *Au, const float *z, float *r, double *part) {
    __shared__ double sd[32];
    double s = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float v = Au[i] - z[i];
        r[i] = v;
        s += (double)v * v;
    }
    s = block_sum1(s, sd);
    if (threadIdx.x == 0)
        part[blockIdx.x] += s;
}

// dL/dm_pq += scale * (A^T r)_p z[q] on A's pattern (probes one at a time,
// so the accumulation order over probes is fixed).
__global__ void k_grad_m(int n, const int *rowptr, const int *colind, const float *atr,
                         const float *z, float scale, float *gm, int first) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float a = atr[p] * scale;
        for (int k = rowptr[p]; k < rowptr[p + 1]; ++k) {
            const float v = a * z[colind[k]];
            gm[k] = first ? v : gm[k] + v;
        }
    }
}

// Sum of the per-block loss partials (fixed order) into out[0].
__global__ void k_sum_parts(int nb, const double *part, double scale, double *out) {
    __shared__ double sd[32];
    double s = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        s += part[b];
    s = block_sum1(s, sd);
    if (threadIdx.x == 0)
        out[0] = s * scale;
}

// Backward through the MLP and the weight-gradient contractions, tile by tile
// (TK nonzeros): D2 = dg w3 [H2 > 0], D1 = [H1 > 0] (D2 W2), then
// dW2 += D2^T H1, dW1 += D1^T F, db1 += sum D1, db2 += sum D2,
// dw3 += sum dg H2, db3 += sum dg.  dg = dL/dm * (1/d_p).  Each block keeps
// its share of the 4801 sums in registers and writes them once; the last
// block reduces the partials in block order.
__global__ void __launch_bounds__(BWD_THREADS) k_mlp_bwd(int64_t nnz, const float *feat,
                                                         const float *params, const float *H1,
                                                         const float *H2, const float *gm,
                                                         float *part, unsigned *counter,
                                                         float *grad) {
    extern __shared__ __align__(16) float sm[];
    float *sW2 = sm;                       // NH * NH
    float *sw3 = sW2 + NH * NH;            // NH
    float *H1t = sw3 + NH;                 // NH * TKP
    float *H2t = H1t + NH * TKP;           // NH * TKP
    float *D2t = H2t + NH * TKP;           // NH * TKP
    float *D1t = D2t + NH * TKP;           // NH * TKP
    float *Ft = D1t + NH * TKP;            // NF * TKP
    float *dgt = Ft + NF * TKP;            // TK
    const int tid = threadIdx.x;
    for (int i = tid; i < NH * NH; i += BWD_THREADS)
        sW2[i] = params[P_W2 + i];
    for (int i = tid; i < NH; i += BWD_THREADS)
        sw3[i] = params[P_W3 + i];
    // thread-owned sums
    const int o_own = tid >> 2, i_own0 = (tid & 3) * 16;  // dW2[o_own][i_own0 .. +15]
    const int w1_i = tid >> 2, w1_j0 = (tid & 3) * 2;     // dW1[w1_i][w1_j0 .. +1]
    float aW2[16], aW1[2], aV = 0.f;                       // aV: db1 / db2 / dw3 / db3
#pragma unroll
    for (int q = 0; q < 16; ++q)
        aW2[q] = 0.f;
    aW1[0] = aW1[1] = 0.f;
    __syncthreads();
    const int64_t ntiles = (nnz + TK - 1) / TK;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t k0 = tile * TK;
        for (int t = tid; t < TK; t += BWD_THREADS) {
            const int64_t k = k0 + t;
            dgt[t] = (k < nnz) ? gm[k] * feat[8 * nnz + k] : 0.f;
        }
        __syncthreads();
        for (int idx = tid; idx < NH * TK; idx += BWD_THREADS) {
            const int o = idx / TK, t = idx % TK;
            const int64_t k = k0 + t;
            const float h1 = (k < nnz) ? H1[o * nnz + k] : 0.f;
            const float h2 = (k < nnz) ? H2[o * nnz + k] : 0.f;
            H1t[o * TKP + t] = h1;
            H2t[o * TKP + t] = h2;
            D2t[o * TKP + t] = (h2 > 0.f) ? dgt[t] * sw3[o] : 0.f;
        }
        for (int idx = tid; idx < NF * TK; idx += BWD_THREADS) {
            const int j = idx / TK, t = idx % TK;
            const int64_t k = k0 + t;
            Ft[j * TKP + t] = (k < nnz) ? feat[j * nnz + k] : 0.f;
        }
        __syncthreads();
        // D1[i][t] = [H1 > 0] sum_o W2[o][i] D2[o][t]; thread: t = tid % TK, 16 i's
        {
            const int t = tid % TK, ig = (tid / TK) * 16;
            float a[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                a[q] = 0.f;
            for (int o = 0; o < NH; ++o) {
                const float d2 = D2t[o * TKP + t];
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    a[q] += sW2[o * NH + ig + q] * d2;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q)
                D1t[(ig + q) * TKP + t] = (H1t[(ig + q) * TKP + t] > 0.f) ? a[q] : 0.f;
        }
        __syncthreads();
        // weight-gradient contractions over the tile
        for (int t = 0; t < TK; ++t) {
            const float d2 = D2t[o_own * TKP + t];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                aW2[q] += d2 * H1t[(i_own0 + q) * TKP + t];
            const float d1 = D1t[w1_i * TKP + t];
            aW1[0] += d1 * Ft[w1_j0 * TKP + t];
            aW1[1] += d1 * Ft[(w1_j0 + 1) * TKP + t];
        }
        if (tid < NH) {
            for (int t = 0; t < TK; ++t)
                aV += D1t[tid * TKP + t];
        } else if (tid < 2 * NH) {
            for (int t = 0; t < TK; ++t)
                aV += D2t[(tid - NH) * TKP + t];
        } else if (tid < 3 * NH) {
            for (int t = 0; t < TK; ++t)
                aV += dgt[t] * H2t[(tid - 2 * NH) * TKP + t];
        } else if (tid == 3 * NH) {
            for (int t = 0; t < TK; ++t)
                aV += dgt[t];
        }
        __syncthreads();
    }
    float *mine = part + (size_t)blockIdx.x * NPARAM;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        mine[P_W2 + o_own * NH + i_own0 + q] = aW2[q];
    mine[P_W1 + w1_i * NF + w1_j0] = aW1[0];
    mine[P_W1 + w1_i * NF + w1_j0 + 1] = aW1[1];
    if (tid < NH)
        mine[P_B1 + tid] = aV;
    else if (tid < 2 * NH)
        mine[P_B2 + tid - NH] = aV;
    else if (tid < 3 * NH)
        mine[P_W3 + tid - 2 * NH] = aV;
    else if (tid == 3 * NH)
        mine[P_B3] = aV;
    if (!arrive_last(counter))
        return;
    for (int i = tid; i < NPARAM; i += BWD_THREADS) {
        float s = 0.f;
        for (int b = 0; b < (int)gridDim.x; ++b)
            s += ldcg(part + (size_t)b * NPARAM + i);
        grad[i] = s;
    }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  The factors
// (1 - b), and the bias corrections come from the host in binary64 rounded
// once to binary32 (forming 1 - b2 from a rounded b2 would lose ~1e-5).
__global__ void k_adam(int np, float *p, float *m, float *v, const float *g, float lr, float b1,
                       float omb1, float b2, float omb2, float c1, float c2, float eps) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + omb1 * gi;
        const float vi = b2 * v[i] + omb2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Rademacher probes z_p[i] = +-1 from a counter-based 64-bit mix of
// (seed, p, i) (the splitmix64 finaliser of Steele, Lea and Flood).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_rademacher(int n, int P, uint64_t seed, float *Z) {
    const int64_t total = (int64_t)n * P;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x)
        Z[idx] = (mix64(seed ^ mix64((uint64_t)idx)) >> 63) ? 1.f : -1.f;
}

__global__ void k_cast_f32(int64_t cnt, const double *a, float *b) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] = (float)a[k];
}

size_t bwd_smem() {
    return sizeof(float) * (NH * NH + NH + 4 * NH * TKP + NF * TKP + TK);
}

// Transpose of A (host-side from the device copy) when the handle lacks it.
gmres_status ensure_transpose(gmres_handle *h) {
    if (h->trowptr.p)
        return GMRES_OK;
    const int n = h->n;
    const int64_t nnz = h->nnz;
    std::vector<int32_t> rp(n + 1), ci(nnz), trp(n + 1, 0), tci(nnz);
    std::vector<double> va(nnz), tva(nnz);
    CK(cudaMemcpy(rp.data(), h->rowptr.p, 4 * (n + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ci.data(), h->colind.p, 4 * nnz, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(va.data(), h->vals64.p, 8 * nnz, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nnz; ++k)
        trp[ci[k] + 1]++;
    for (int i = 0; i < n; ++i)
        trp[i + 1] += trp[i];
    std::vector<int32_t> pos(trp.begin(), trp.end() - 1);
    for (int i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t d = pos[ci[k]]++;
            tci[d] = i;
            tva[d] = va[k];
        }
    CK(h->trowptr.ensure(4 * (n + 1)));
    CK(h->tcolind.ensure(4 * std::max<int64_t>(nnz, 1)));
    CK(h->tvals64.ensure(8 * std::max<int64_t>(nnz, 1)));
    CK(cudaMemcpy(h->trowptr.p, trp.data(), 4 * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->tcolind.p, tci.data(), 4 * nnz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->tvals64.p, tva.data(), 8 * nnz, cudaMemcpyHostToDevice));
    return GMRES_OK;
}

// Features of the current matrix (cached until the values change).
gmres_status ensure_features(gmres_handle *h) {
    if (h->spai_feat_ok)
        return GMRES_OK;
    gmres_status st = ensure_transpose(h);
    if (st != GMRES_OK)
        return st;
    const int n = h->n;
    const int64_t nnz = h->nnz;
    CK(h->spai_feat.ensure(sizeof(float) * 9 * std::max<int64_t>(nnz, 1)));
    CK(h->spai_rowv.ensure(sizeof(float) * 3 * n));
    CK(h->tvals32.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)));
    float *dinv = h->spai_rowv.as<float>(), *rowabs = dinv + n, *colabs = rowabs + n;
    const int g = h->nsm * 4;
    k_rowstats<<<g, 256, 0, h->stream>>>(n, h->rowptr.as<int>(), h->colind.as<int>(),
                                         h->vals64.as<double>(), dinv, rowabs);
    k_colstats<<<g, 256, 0, h->stream>>>(n, h->trowptr.as<int>(), h->tvals64.as<double>(), dinv,
                                         colabs);
    k_features<<<g, 256, 0, h->stream>>>(n, nnz, h->rowptr.as<int>(), h->colind.as<int>(),
                                         h->vals64.as<double>(), dinv, rowabs, colabs,
                                         h->spai_feat.as<float>());
    k_cast_f32<<<g, 256, 0, h->stream>>>(nnz, h->tvals64.as<double>(), h->tvals32.as<float>());
    CKL();
    h->spai_feat_ok = 1;
    return GMRES_OK;
}

template <class F>
gmres_status with_params(gmres_handle *h, const float *params, F &&fn) {
    const float *dp = params;
    if (!is_device_ptr(params)) {
        CK(h->spai_params.ensure(sizeof(float) * NPARAM));
        CK(cudaMemcpyAsync(h->spai_params.p, params, sizeof(float) * NPARAM,
                           cudaMemcpyHostToDevice, h->stream));
        dp = h->spai_params.as<float>();
    }
    return fn(dp);
}

// Loss and gradients for probes Z (device, n x P column-major, binary32).
gmres_status loss_grad(gmres_handle *h, const float *params, int P, const float *Z, double *loss,
                       float *grad_params, float *grad_m_out) {
    gmres_status st = ensure_features(h);
    if (st != GMRES_OK)
        return st;
    const int n = h->n;
    const int64_t nnz = h->nnz;
    const int g = h->nsm * 4;
    CK(h->spai_m.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)));
    CK(h->spai_gm.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)));
    CK(h->spai_H.ensure(sizeof(float) * 2 * NH * std::max<int64_t>(nnz, 1)));
    CK(h->spai_vec.ensure(sizeof(float) * 3 * (size_t)n));
    CK(h->spai_part.ensure(sizeof(float) * (size_t)h->nsm * 2 * NPARAM + 8 * (g + 2)));
    float *m = h->spai_m.as<float>(), *gm = h->spai_gm.as<float>();
    float *H1 = h->spai_H.as<float>(), *H2 = H1 + (size_t)NH * nnz;
    float *u = h->spai_vec.as<float>(), *au = u + n, *r = au + n;
    float *wpart = h->spai_part.as<float>();
    double *lpart = reinterpret_cast<double *>(wpart + (size_t)h->nsm * 2 * NPARAM);
    k_mlp_fwd<<<g, 256, 0, h->stream>>>(nnz, h->spai_feat.as<float>(), params, m, nullptr, H1,
                                        H2);
    CKL();
    CK(cudaMemsetAsync(lpart, 0, sizeof(double) * (g + 2), h->stream));
    const int L = h->lanes32;
    const int *rp = h->rowptr.as<int>(), *ci = h->colind.as<int>();
    const float scale = (float)(1.0 / ((double)P * (double)n));
    for (int p = 0; p < P; ++p) {
        const float *z = Z + (size_t)p * n;
        // u = M z, r = A u - z, atr = A^T r
        {
            dim3 gg(h->nsm * 8), bb(256);
            switch (L) {
            case 1: k_spmv_plain<float, float, 1><<<gg, bb, 0, h->stream>>>(n, rp, ci, m, z, u); break;
            case 2: k_spmv_plain<float, float, 2><<<gg, bb, 0, h->stream>>>(n, rp, ci, m, z, u); break;
            case 4: k_spmv_plain<float, float, 4><<<gg, bb, 0, h->stream>>>(n, rp, ci, m, z, u); break;
            case 8: k_spmv_plain<float, float, 8><<<gg, bb, 0, h->stream>>>(n, rp, ci, m, z, u); break;
            default: k_spmv_plain<float, float, 16><<<gg, bb, 0, h->stream>>>(n, rp, ci, m, z, u); break;
            }
            k_spmv_plain<float, float, 4><<<gg, bb, 0, h->stream>>>(n, rp, ci, h->vals32.as<float>(), u,
                                                              au);
            k_probe_residual<<<g, 256, 0, h->stream>>>(n, au, z, r, lpart);
            k_spmv_plain<float, float, 4><<<gg, bb, 0, h->stream>>>(
                n, h->trowptr.as<int>(), h->tcolind.as<int>(), h->tvals32.as<float>(), r, au);
            k_grad_m<<<g, 256, 0, h->stream>>>(n, rp, ci, au, z, scale, gm, p == 0);
        }
        CKL();
    }
    k_sum_parts<<<1, 256, 0, h->stream>>>(g, lpart, 0.5 * (double)scale, lpart + g);
    CKL();
    if (grad_params) {
        const size_t smb = bwd_smem();
        static bool attr = false;
        if (!attr) {
            CK(cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smb));
            attr = true;
        }
        CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream));
        const int gb = h->nsm * 2;
        k_mlp_bwd<<<gb, BWD_THREADS, smb, h->stream>>>(
            nnz, h->spai_feat.as<float>(), params, H1, H2, gm, wpart,
            &h->ctl.as<Ctl>()->counter[7], grad_params);
        CKL();
    }
    if (grad_m_out)
        CK(cudaMemcpyAsync(grad_m_out, gm, sizeof(float) * nnz, cudaMemcpyDeviceToDevice,
                           h->stream));
    if (loss)
        CK(cudaMemcpyAsync(loss, lpart + g, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

gmres_status prepare(gmres_handle *h) {
    if (!h || h->split)  // the preconditioner works on the binary64 + binary32 copies
        return GMRES_ERR_ARG;
    // the control block is used for the last-block counter
    CK(h->ctl.ensure(sizeof(Ctl)));
    return GMRES_OK;
}

}  // namespace

extern "C" {

gmres_status gmres_spai_features(gmres_t h, float *feat) {
    gmres_status st = prepare(h);
    if (st != GMRES_OK)
        return st;
    st = ensure_features(h);
    if (st != GMRES_OK)
        return st;
    if (feat) {
        if (is_device_ptr(feat))
            CK(cudaMemcpyAsync(feat, h->spai_feat.p, sizeof(float) * 8 * h->nnz,
                               cudaMemcpyDeviceToDevice, h->stream));
        else
            CK(cudaMemcpyAsync(feat, h->spai_feat.p, sizeof(float) * 8 * h->nnz,
                               cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

gmres_status gmres_spai_loss_grad(gmres_t h, const float *params, int32_t nprobe, const float *Z,
                                  double *loss, float *grad_params, float *grad_m) {
    if (!h || h->split || !params || nprobe < 1 || !Z || !is_device_ptr(Z) ||
        (grad_params && !is_device_ptr(grad_params)) || (grad_m && !is_device_ptr(grad_m)))
        return GMRES_ERR_ARG;
    gmres_status st = prepare(h);
    if (st != GMRES_OK)
        return st;
    return with_params(h, params, [&](const float *dp) {
        return loss_grad(h, dp, nprobe, Z, loss, grad_params, grad_m);
    });
}

gmres_status gmres_spai_adam(gmres_t h, float *params, float *adam_m, float *adam_v,
                             const float *grad, int32_t step, float lr) {
    if (!h || !params || !adam_m || !adam_v || !grad || step < 1 || !(lr > 0) ||
        !is_device_ptr(params) || !is_device_ptr(adam_m) || !is_device_ptr(adam_v) ||
        !is_device_ptr(grad))
        return GMRES_ERR_ARG;
    const double b1 = 0.9, b2 = 0.999;
    k_adam<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(
        NPARAM, params, adam_m, adam_v, grad, lr, (float)b1, (float)(1.0 - b1), (float)b2,
        (float)(1.0 - b2), (float)(1.0 - std::pow(b1, step)), (float)(1.0 - std::pow(b2, step)),
        1e-8f);
    CKL();
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

gmres_status gmres_spai_train_step(gmres_t h, float *params, float *adam_m, float *adam_v,
                                   int32_t step, int32_t nprobe, uint64_t seed, const float *Zx,
                                   int32_t nzx, float lr, double *loss) {
    if (!h || h->split || !params || !adam_m || !adam_v || step < 1 || nprobe < 0 || nzx < 0 ||
        nprobe + nzx < 1 || (nzx > 0 && (!Zx || !is_device_ptr(Zx))) || !is_device_ptr(params) ||
        !is_device_ptr(adam_m) || !is_device_ptr(adam_v) || !(lr > 0))
        return GMRES_ERR_ARG;
    gmres_status st = prepare(h);
    if (st != GMRES_OK)
        return st;
    const int n = h->n, P = nprobe + nzx;
    CK(h->spai_Z.ensure(sizeof(float) * (size_t)n * P));
    CK(h->spai_grad.ensure(sizeof(float) * NPARAM));
    float *Z = h->spai_Z.as<float>();
    if (nprobe > 0) {
        k_rademacher<<<h->nsm * 4, 256, 0, h->stream>>>(n, nprobe, seed, Z);
        CKL();
    }
    if (nzx > 0)
        CK(cudaMemcpyAsync(Z + (size_t)n * nprobe, Zx, sizeof(float) * (size_t)n * nzx,
                           cudaMemcpyDeviceToDevice, h->stream));
    st = loss_grad(h, params, P, Z, loss, h->spai_grad.as<float>(), nullptr);
    if (st != GMRES_OK)
        return st;
    return gmres_spai_adam(h, params, adam_m, adam_v, h->spai_grad.as<float>(), step, lr);
}

gmres_status gmres_spai_set(gmres_t h, const float *params) {
    if (!h || !params)
        return GMRES_ERR_ARG;
    gmres_status st = prepare(h);
    if (st != GMRES_OK)
        return st;
    st = ensure_features(h);
    if (st != GMRES_OK)
        return st;
    const int64_t nnz = h->nnz;
    CK(h->pvals32.ensure(sizeof(float) * std::max<int64_t>(nnz, 1)));
    CK(h->pvals64.ensure(sizeof(double) * std::max<int64_t>(nnz, 1)));
    st = with_params(h, params, [&](const float *dp) {
        k_mlp_fwd<<<h->nsm * 8, 256, 0, h->stream>>>(nnz, h->spai_feat.as<float>(), dp,
                                                     h->pvals32.as<float>(),
                                                     h->pvals64.as<double>(), nullptr, nullptr);
        CKL();
        return GMRES_OK;
    });
    if (st != GMRES_OK)
        return st;
    CK(cudaStreamSynchronize(h->stream));
    h->has_precond = 1;
    return GMRES_OK;
}

gmres_status gmres_spai_values(gmres_t h, double *mvals) {
    if (!h || !mvals || !h->has_precond)
        return GMRES_ERR_ARG;
    CK(cudaMemcpyAsync(mvals, h->pvals64.p, sizeof(double) * h->nnz,
                       is_device_ptr(mvals) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return GMRES_OK;
}

gmres_status gmres_spai_clear(gmres_t h) {
    if (!h)
        return GMRES_ERR_ARG;
    h->has_precond = 0;
    return GMRES_OK;
}

}  // extern "C"
