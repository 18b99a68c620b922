// Reverse mode (adjoint) of a shared-step Hermite rollout: the predictor and
// corrector of Sect. 2 of Portegies Zwart, Belleman & Geldof (2007) are
// linear in (x, v, a, k, a_p, k_p), so their adjoints are their transposes;
// the force of Eq. (Force) with the Appendix A pair term needs a vector-
// Jacobian product, evaluated here in FP32 pair arithmetic like the forward
// force, with FP64 totals.  With R = (eps^2 + |d|^2)^(-1/2), d = x_j - x_i,
// e = v_j - v_i, the pair (i, j) sends to x_j (and minus it to x_i)
//   m_j [R^3 g_a - 3 R^5 (d.g_a) d]
//     + m_j [-3 R^5 (e.g_k) d - 3 R^5 (d.g_k) e + 15 R^7 (d.e)(d.g_k) d - 3 R^5 (d.e) g_k],
// to v_j (minus to v_i) m_j [R^3 g_k - 3 R^5 (d.g_k) d], and to m_j
// R^3 (d.g_a) + R^3 (e.g_k) - 3 R^5 (d.e)(d.g_k), where (g_a, g_k) are the
// upstream gradients of particle i's acceleration and jerk.  For one particle
// p both of its roles combine linearly: with G_a = m_p g_a,q - m_q g_a,p and
// G_k likewise, one evaluation per pair (p, q) gives p's position and
// velocity gradients.
#include "force_impl.cuh"  // fold_ds_rn; nbody_internal.cuh, ptx.cuh

namespace nb {

namespace {

constexpr int kVjpThreads = 128;
constexpr int kVjpTile = 128;

// grid (i-blocks, j-ranges): block (x, y) takes the particles p of i-block x
// against the j-tiles of range y.  With one range it adds its totals to the
// gradients; with several it writes them to part[y][7][n] and
// vjp_reduce_kernel adds the ranges in ascending order (deterministic).
__global__ void __launch_bounds__(kVjpThreads)
    force_vjp_kernel(const float4 *__restrict__ posm, const float4 *__restrict__ vel,
                     const float4 *__restrict__ gA, const float4 *__restrict__ gK, int n, int n_pad, float eps2,
                     int tiles_per_range, double *__restrict__ part, DiffGrads G)
{
    __shared__ float4 sp[kVjpTile], sv[kVjpTile], sa[kVjpTile], sk[kVjpTile];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int pl = p < n ? p : 0;
    const float4 xi = posm[pl], vi = vel[pl], ga = gA[pl], gk = gK[pl];
    const float mp = xi.w;
    // running totals over the tiles as double-single pairs on the FP32 pipe (fold_ds_rn;
    // GB300's FP64 unit takes ~19 cycles per warp instruction), hi + lo in FP64 at the end
    float hx[3] = {0, 0, 0}, lx[3] = {0, 0, 0}, hv[3] = {0, 0, 0}, lv[3] = {0, 0, 0}, hm = 0.f, lm = 0.f;
    const int j_begin = blockIdx.y * tiles_per_range * kVjpTile;
    const int j_end = min(j_begin + tiles_per_range * kVjpTile, n_pad);
    for (int j0 = j_begin; j0 < j_end; j0 += kVjpTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kVjpTile; t += blockDim.x) {
            sp[t] = posm[j0 + t];
            sv[t] = vel[j0 + t];
            sa[t] = gA[j0 + t];
            sk[t] = gK[j0 + t];
        }
        __syncthreads();
        float px[3] = {0, 0, 0}, pv[3] = {0, 0, 0}, pm = 0.f;
#pragma unroll 4
        for (int t = 0; t < kVjpTile; ++t) {
            const float4 xq = sp[t], vq = sv[t], gaq = sa[t], gkq = sk[t];
            const float mq = xq.w;
            const float d0 = xi.x - xq.x, d1 = xi.y - xq.y, d2 = xi.z - xq.z;  // d = x_p - x_q
            const float e0 = vi.x - vq.x, e1 = vi.y - vq.y, e2 = vi.z - vq.z;
            const float r2 = fmaf(d2, d2, fmaf(d1, d1, fmaf(d0, d0, eps2)));
            const float R = rsqrt_mufu(r2);
            const float R2 = R * R, R3 = R2 * R, R5 = R3 * R2, R7 = R5 * R2;
            const float A0 = fmaf(-mq, ga.x, mp * gaq.x), A1 = fmaf(-mq, ga.y, mp * gaq.y),
                        A2 = fmaf(-mq, ga.z, mp * gaq.z);
            const float K0 = fmaf(-mq, gk.x, mp * gkq.x), K1 = fmaf(-mq, gk.y, mp * gkq.y),
                        K2 = fmaf(-mq, gk.z, mp * gkq.z);
            const float dA = fmaf(d2, A2, fmaf(d1, A1, d0 * A0));
            const float eK = fmaf(e2, K2, fmaf(e1, K1, e0 * K0));
            const float dK = fmaf(d2, K2, fmaf(d1, K1, d0 * K0));
            const float de = fmaf(d2, e2, fmaf(d1, e1, d0 * e0));
            const float cd = fmaf(15.0f * R7 * de, dK, -3.0f * R5 * (dA + eK));
            const float ce = -3.0f * R5 * dK;
            const float cg = -3.0f * R5 * de;
            px[0] += fmaf(cg, K0, fmaf(ce, e0, fmaf(cd, d0, R3 * A0)));
            px[1] += fmaf(cg, K1, fmaf(ce, e1, fmaf(cd, d1, R3 * A1)));
            px[2] += fmaf(cg, K2, fmaf(ce, e2, fmaf(cd, d2, R3 * A2)));
            pv[0] += fmaf(ce, d0, R3 * K0);
            pv[1] += fmaf(ce, d1, R3 * K1);
            pv[2] += fmaf(ce, d2, R3 * K2);
            // p as the source of q's force: d . g_a,q etc.
            const float dga = fmaf(d2, gaq.z, fmaf(d1, gaq.y, d0 * gaq.x));
            const float egk = fmaf(e2, gkq.z, fmaf(e1, gkq.y, e0 * gkq.x));
            const float dgk = fmaf(d2, gkq.z, fmaf(d1, gkq.y, d0 * gkq.x));
            pm += fmaf(R3, dga + egk, -3.0f * R5 * de * dgk);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            fold_ds_rn(hx[c], lx[c], px[c]);
            fold_ds_rn(hv[c], lv[c], pv[c]);
        }
        fold_ds_rn(hm, lm, pm);
    }
    if (p >= n) return;
    double tx[3], tv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        tx[c] = static_cast<double>(hx[c]) + static_cast<double>(lx[c]);
        tv[c] = static_cast<double>(hv[c]) + static_cast<double>(lv[c]);
    }
    const double tm = static_cast<double>(hm) + static_cast<double>(lm);
    if (gridDim.y == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            G.gxp[c][p] += tx[c];
            G.gvp[c][p] += tv[c];
        }
        G.gm[p] += tm;
    } else {
        double *b = part + static_cast<size_t>(blockIdx.y) * 7 * n + p;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            b[static_cast<size_t>(c) * n] = tx[c];
            b[static_cast<size_t>(3 + c) * n] = tv[c];
        }
        b[static_cast<size_t>(6) * n] = tm;
    }
}

// One thread per (particle, component): adds the component's ranges in order.
__global__ void vjp_reduce_kernel(const double *__restrict__ part, int ranges, int n, DiffGrads G)
{
    const int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (idx >= 7LL * n) return;
    const int c = static_cast<int>(idx / n);
    const int p = static_cast<int>(idx - static_cast<int64_t>(c) * n);
    double t = 0.0;
    for (int y = 0; y < ranges; ++y) t += part[(static_cast<size_t>(y) * 7 + c) * n + p];
    if (c < 3)
        G.gxp[c][p] += t;
    else if (c < 6)
        G.gvp[c - 3][p] += t;
    else
        G.gm[p] += t;
}

// Transposed corrector: from the gradients of the corrected state (gx, gv, ga,
// gk) to those of the predicted state (gxp, gvp), of the force (gA, gK, FP32)
// and of the start-of-step a, k (left in ga, gk).
__global__ void adj_correct_kernel(DiffGrads G, int n, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c1 = dt * dt * dt * dt / 24.0, c2 = dt * dt * dt * dt * dt / 120.0;
    const double c3 = dt * dt * dt / 6.0, c4 = dt * dt * dt * dt / 24.0;
    float ap[3], kp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double gx = G.gx[c][i], gv = G.gv[c][i];
        const double g2 = c1 * gx + c3 * gv, g3 = c2 * gx + c4 * gv;
        ap[c] = static_cast<float>(6.0 / (dt * dt) * g2 - 12.0 / (dt * dt * dt) * g3 + G.ga[c][i]);
        kp[c] = static_cast<float>(-2.0 / dt * g2 + 6.0 / (dt * dt) * g3 + G.gk[c][i]);
        G.ga[c][i] = -6.0 / (dt * dt) * g2 + 12.0 / (dt * dt * dt) * g3;
        G.gk[c][i] = -4.0 / dt * g2 + 6.0 / (dt * dt) * g3;
        G.gxp[c][i] = gx;
        G.gvp[c][i] = gv;
    }
    G.gA[i] = make_float4(ap[0], ap[1], ap[2], 0.f);
    G.gK[i] = make_float4(kp[0], kp[1], kp[2], 0.f);
}

// Transposed predictor: gradients of the start-of-step state.
__global__ void adj_predict_kernel(DiffGrads G, int n, double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double gxp = G.gxp[c][i], gvp = G.gvp[c][i];
        G.gx[c][i] = gxp;
        G.gv[c][i] = gxp * dt + gvp;
        G.ga[c][i] += gxp * dt * dt / 2.0 + gvp * dt;
        G.gk[c][i] += gxp * dt * dt * dt / 6.0 + gvp * dt * dt / 2.0;
    }
}

// Start of the rollout: the upstream of the t = 0 force is (ga, gk) itself.
__global__ void adj_init_kernel(DiffGrads G, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float ap[3], kp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ap[c] = static_cast<float>(G.ga[c][i]);
        kp[c] = static_cast<float>(G.gk[c][i]);
        G.gxp[c][i] = G.gx[c][i];
        G.gvp[c][i] = G.gv[c][i];
    }
    G.gA[i] = make_float4(ap[0], ap[1], ap[2], 0.f);
    G.gK[i] = make_float4(kp[0], kp[1], kp[2], 0.f);
}

// Loss L = sum |x|^2 + E_pot (FP64) and its gradient at the final state:
// dL/dx_i = 2 x_i - m_i a_i, dL/dm_i = phi_i; per-particle loss terms in lval.
__global__ void loss_kernel(const State S, double eps2, DiffGrads G, double *__restrict__ lval)
{
    __shared__ double sx[128], sy[128], sz[128], sm[128];
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const bool live = i < S.n;
    const double xi = live ? S.x[0][i] : 0.0, yi = live ? S.x[1][i] : 0.0, zi = live ? S.x[2][i] : 0.0;
    double phi = 0.0, a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t j0 = 0; j0 < S.n; j0 += 128) {
        __syncthreads();
        for (int t = threadIdx.x; t < 128; t += blockDim.x) {
            const int64_t j = j0 + t;
            const bool ok = j < S.n;
            sx[t] = ok ? S.x[0][j] : 0.0;
            sy[t] = ok ? S.x[1][j] : 0.0;
            sz[t] = ok ? S.x[2][j] : 0.0;
            sm[t] = ok ? S.m[j] : 0.0;
        }
        __syncthreads();
        const int jn = static_cast<int>(S.n - j0 < 128 ? S.n - j0 : 128);
        for (int t = 0; t < jn; ++t) {
            if (j0 + t == i) continue;
            const double dx = sx[t] - xi, dy = sy[t] - yi, dz = sz[t] - zi;
            const double r2 = eps2 + dx * dx + dy * dy + dz * dz;
            const double rinv = 1.0 / sqrt(r2);
            const double r3 = rinv * rinv * rinv;
            phi -= sm[t] * rinv;
            a0 += sm[t] * dx * r3;
            a1 += sm[t] * dy * r3;
            a2 += sm[t] * dz * r3;
        }
    }
    if (!live) return;
    const double mi = S.m[i];
    G.gx[0][i] = 2.0 * xi - mi * a0;
    G.gx[1][i] = 2.0 * yi - mi * a1;
    G.gx[2][i] = 2.0 * zi - mi * a2;
    G.gm[i] = phi;
    lval[i] = xi * xi + yi * yi + zi * zi + 0.5 * mi * phi;
}

__global__ void sum_kernel(const double *__restrict__ v, int64_t n, double *out)
{
    __shared__ double s[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (static_cast<int>(threadIdx.x) < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// Shared step: every particle's time is `tick` and level `level`.
__global__ void set_time_kernel(const State S, int64_t tick, int level)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < S.n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        S.t[i] = tick;
        S.level[i] = static_cast<int8_t>(level);
    }
}

int blocks_of(int64_t n, int t) { return static_cast<int>((n + t - 1) / t); }

}  // namespace

int vjp_ranges(int64_t n, int64_t n_pad, int sm_count)
{
    // enough blocks for about four per SM; ranges of whole tiles
    const int bx = blocks_of(n, kVjpThreads);
    const int tiles = static_cast<int>(n_pad / kVjpTile);
    const int want = (4 * sm_count + bx - 1) / bx;
    const int r = want < 1 ? 1 : (want > tiles ? tiles : want);
    const int tpr = (tiles + r - 1) / r;
    return (tiles + tpr - 1) / tpr;
}

size_t vjp_scratch_doubles(int64_t n, int64_t n_pad, int sm_count)
{
    const int r = vjp_ranges(n, n_pad, sm_count);
    return r > 1 ? static_cast<size_t>(r) * 7 * static_cast<size_t>(n) : 0;
}

cudaError_t force_vjp_launch(const JStream &J, const DiffGrads &G, int64_t n, float eps2, int sm_count,
                             double *scratch, cudaStream_t s, int64_t *launches)
{
    const int tiles = static_cast<int>(J.n_pad / kVjpTile);
    const int r = vjp_ranges(n, J.n_pad, sm_count);
    const int tpr = (tiles + r - 1) / r;
    const dim3 grid(blocks_of(n, kVjpThreads), r);
    force_vjp_kernel<<<grid, kVjpThreads, 0, s>>>(J.posm, J.vel, G.gA, G.gK, static_cast<int>(n),
                                                  static_cast<int>(J.n_pad), eps2, tpr, scratch, G);
    ++*launches;
    if (r > 1) {
        vjp_reduce_kernel<<<blocks_of(7 * n, 256), 256, 0, s>>>(scratch, r, static_cast<int>(n), G);
        ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t adj_correct_launch(const DiffGrads &G, int64_t n, double dt, cudaStream_t s, int64_t *launches)
{
    const int t = n >= 152 * 256 ? 256 : 32;  // FP64-heavy rows: spread small n over more SMs
    adj_correct_kernel<<<blocks_of(n, t), t, 0, s>>>(G, static_cast<int>(n), dt);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t adj_predict_launch(const DiffGrads &G, int64_t n, double dt, cudaStream_t s, int64_t *launches)
{
    const int t = n >= 152 * 256 ? 256 : 32;
    adj_predict_kernel<<<blocks_of(n, t), t, 0, s>>>(G, static_cast<int>(n), dt);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t adj_init_launch(const DiffGrads &G, int64_t n, cudaStream_t s, int64_t *launches)
{
    adj_init_kernel<<<blocks_of(n, 256), 256, 0, s>>>(G, static_cast<int>(n));
    ++*launches;
    return cudaGetLastError();
}

cudaError_t loss_launch(const State &S, double eps2, const DiffGrads &G, double *lval, double *loss, cudaStream_t s,
                        int64_t *launches)
{
    loss_kernel<<<blocks_of(S.n, 128), 128, 0, s>>>(S, eps2, G, lval);
    sum_kernel<<<1, 1024, 0, s>>>(lval, S.n, loss);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t set_time_launch(const State &S, int64_t tick, int level, cudaStream_t s, int64_t *launches)
{
    set_time_kernel<<<blocks_of(S.n, 256) < 1024 ? blocks_of(S.n, 256) : 1024, 256, 0, s>>>(S, tick, level);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace nb
