// K3: sgn(H_k) e_1 by Roberts' iteration S <- (S + S^-1)/2, S^0 = H_k
// (Sec. 5.2, Eq. Roberts; used for H_k in Sec. 5.3 step v), in FP64 on the
// device: a thread-block cluster (one block per SM) per right-hand side
// while the matrix fits the cluster's shared memory (k up to about 320), one
// thread block per right-hand side above. The cluster size (4 to 8) is
// chosen at launch so that the clusters of all right-hand sides are resident
// in as few waves as possible.
//
// The inverse is an in-place Gauss-Jordan elimination with partial (row)
// pivoting; the row interchanges are undone as column interchanges at the
// end. Stopping rule: after the first iterate whose relative change
// ||S^(n+1) - S^n||_F / ||S^(n+1)||_F is <= 1e-9, one more iteration (the
// quadratic convergence then reaches rounding level); at most 50 iterations.
// A zero or non-finite pivot (an eigenvalue on or numerically at the
// imaginary axis makes S singular) ends with status OVS_ESIGN; no
// convergence within 50 iterations gives OVS_NOT_CONVERGED.
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace ovs {

constexpr int NT = 1024;
constexpr double kSwitchTol = 1e-9;
constexpr int kExtra = 1;
constexpr int kMaxIter = 50;
enum { ST_OK = 0, ST_NOT_CONVERGED = 1, ST_ESIGN = -6 };

__device__ __forceinline__ double blk_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

// In-place inverse of the n x n row-major matrix A. Returns false if a
// pivot is zero or not finite.
__device__ bool gauss_jordan(cd* A, int n, int* perm, cd* colp, cd* rowp, double* sval, int* sidx) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    __shared__ int s_ok;
    __shared__ double2 s_inv;
    if (tid == 0) s_ok = 1;
    for (int p = 0; p < n; ++p) {
        // pivot: argmax_{i >= p} |A[i][p]|
        double best = -1.0;
        int bi = p;
        for (int i = p + tid; i < n; i += NT) {
            const cd a = A[(size_t)i * n + p];
            const double v = a.re * a.re + a.im * a.im;
            if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { sval[w] = best; sidx[w] = bi; }
        __syncthreads();
        if (tid == 0) {
            double b = sval[0];
            int ib = sidx[0];
            for (int q = 1; q < NT / 32; ++q)
                if (sval[q] > b || (sval[q] == b && sidx[q] < ib)) { b = sval[q]; ib = sidx[q]; }
            perm[p] = ib;
            if (!(b > 0.0) || !isfinite(b)) {
                s_ok = 0;
            } else {  // the pivot's inverse, once per block (A[ib][p] is A[p][p] after the swap)
                const cd a = A[(size_t)ib * n + p];
                const double den = a.re * a.re + a.im * a.im;
                s_inv = make_double2(a.re / den, -a.im / den);
            }
        }
        __syncthreads();
        if (!s_ok) return false;
        const int piv = perm[p];
        if (piv != p) {
            for (int j = tid; j < n; j += NT) {
                const cd t = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = A[(size_t)piv * n + j];
                A[(size_t)piv * n + j] = t;
            }
            __syncthreads();
        }
        const cd inv = {s_inv.x, s_inv.y};
        for (int i = tid; i < n; i += NT) {
            colp[i] = A[(size_t)i * n + p];
            rowp[i] = (i == p) ? inv : cmul(A[(size_t)p * n + i], inv);
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += NT) {
            const int i = idx / n, j = idx - i * n;
            if (i == p) {
                A[idx] = rowp[j];
            } else if (j == p) {
                A[idx] = -cmul(colp[i], inv);
            } else {
                cd v = A[idx];
                const cd f = colp[i], g = rowp[j];
                v.re = fma(-f.re, g.re, v.re);
                v.re = fma(f.im, g.im, v.re);
                v.im = fma(-f.re, g.im, v.im);
                v.im = fma(-f.im, g.re, v.im);
                A[idx] = v;
            }
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int p = n - 1; p >= 0; --p) {
        const int q = perm[p];
        if (q != p) {
            for (int i = tid; i < n; i += NT) {
                const cd t = A[(size_t)i * n + p];
                A[(size_t)i * n + p] = A[(size_t)i * n + q];
                A[(size_t)i * n + q] = t;
            }
            __syncthreads();
        }
    }
    return true;
}

__global__ void __launch_bounds__(NT) k_newton(const double2* __restrict__ H, long long h_rhs_stride, int ldh,
                                               const int* __restrict__ k_used, const double* __restrict__ beta,
                                               double2* __restrict__ coeff, long long coeff_stride,
                                               double2* __restrict__ work, int kmax, int* __restrict__ iters,
                                               int* __restrict__ status, const int* __restrict__ active,
                                               int n_fixed) {
    extern __shared__ unsigned char smem_raw[];
    const int r = blockIdx.x, tid = threadIdx.x;
    if (active != nullptr && active[r] == 0) return;
    const int n = n_fixed > 0 ? n_fixed : k_used[r];
    cd* S = reinterpret_cast<cd*>(work) + (size_t)r * 2 * kmax * kmax;
    cd* T = S + (size_t)kmax * kmax;
    cd* colp = reinterpret_cast<cd*>(smem_raw);
    cd* rowp = colp + kmax;
    int* perm = reinterpret_cast<int*>(rowp + kmax);
    __shared__ double sval[NT / 32 + 1];
    __shared__ int sidx[NT / 32];
    double2* cr = coeff + r * coeff_stride;
    if (n <= 0) {
        for (int i = tid; i < kmax; i += NT) cr[i] = make_double2(0.0, 0.0);
        if (tid == 0) { iters[r] = 0; status[r] = ST_OK; }
        return;
    }
    const double2* Hr = H + r * h_rhs_stride;
    for (int idx = tid; idx < n * n; idx += NT) {
        const int i = idx / n, j = idx - i * n;
        const double2 h = Hr[i + (long long)j * ldh];
        S[idx] = {h.x, h.y};
    }
    __syncthreads();
    int st = ST_NOT_CONVERGED, it_done = 0, remaining = -1;
    for (int it = 1; it <= kMaxIter; ++it) {
        for (int idx = tid; idx < n * n; idx += NT) T[idx] = S[idx];
        __syncthreads();
        if (!gauss_jordan(T, n, perm, colp, rowp, sval, sidx)) {
            st = ST_ESIGN;
            it_done = it;
            break;
        }
        double d2 = 0.0, s2 = 0.0;
        for (int idx = tid; idx < n * n; idx += NT) {
            const cd a = S[idx], b = T[idx];
            const cd v = {0.5 * (a.re + b.re), 0.5 * (a.im + b.im)};
            const double dx = v.re - a.re, dy = v.im - a.im;
            d2 += dx * dx + dy * dy;
            s2 += v.re * v.re + v.im * v.im;
            S[idx] = v;
        }
        d2 = blk_sum(d2, sval);
        s2 = blk_sum(s2, sval);
        it_done = it;
        const double change = sqrt(d2 / s2);
        if (!isfinite(change)) {
            st = ST_ESIGN;
            break;
        }
        if (remaining < 0 && change <= kSwitchTol) remaining = kExtra;
        if (remaining >= 0) {
            if (remaining == 0) {
                st = ST_OK;
                break;
            }
            --remaining;
        }
    }
    const double b = beta[r];
    for (int i = tid; i < kmax; i += NT) {
        if (i < n && st != ST_ESIGN) {
            const cd s = S[(size_t)i * n];
            cr[i] = make_double2(b * s.re, b * s.im);
        } else {
            cr[i] = make_double2(0.0, 0.0);
        }
    }
    if (tid == 0) {
        iters[r] = it_done;
        status[r] = st;
    }
}

// ----------------------------------------------------------------------
// Cluster form: one matrix per cluster of ncl CTAs (one per SM; ncl is the
// launch's cluster size). CTA c holds the column block [c*W, c*W + W) of the
// matrix being inverted in shared memory (W = ceil(n/ncl)); the iterate S
// stays in global memory (each CTA touches only its own columns).
//
// Gauss-Jordan with the pivots taken in panels of up to bw consecutive
// columns, all inside one CTA's block (the panel's owner):
//  A. the owner runs the panel's pivots on the panel columns alone: for each
//     pivot p it searches the pivot row, publishes p's pivot row and its
//     (row-swapped) column p, and eliminates on the panel columns;
//  B. one cluster barrier per panel makes the panel visible; every CTA
//     copies it through distributed shared memory and applies the panel's
//     pivots, in order, to all its other columns (swap rows p and pivot,
//     scale the pivot row, eliminate).
// Every column therefore receives the same operations in the same order as
// with one barrier per pivot, so the result is the same bit for bit; the
// cluster barriers and the waits for the pivot search fall by the panel
// width. The published panels are double-buffered by the parity of the
// panel index. After the last panel the row interchanges are undone as a
// column permutation read from the owners' blocks while S <- (S + S^-1)/2
// is formed, and the norms of the change are summed over the cluster.
constexpr int NTC = 512;
constexpr int kMaxPanel = 8;
constexpr int kClusterSizes[] = {8, 7, 6, 5, 4};  // candidates, largest first

__device__ __forceinline__ double cl_block_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < NTC / 32; ++q) s += sh[q];
    __syncthreads();
    return s;
}

// One Gauss-Jordan pivot p on the local columns jj in [jb, je) of T (row
// stride W), skipping the local columns in [sb, se): rows p and piv
// swapped, the pivot row scaled by inv, every other row eliminated with
// the pivot column col (after the swap); column p itself, where present,
// becomes -col * inv with inv on the diagonal. All threads of the CTA call
// it with the same arguments.
__device__ __forceinline__ void gj_apply(cd* T, int W, int n, int c0, int jb, int je, int sb, int se, int p,
                                         int piv, const cd* col, cd inv, cd* rowp) {
    const int tid = threadIdx.x;
    const int w = je - jb;
    if (w <= 0) return;
    if (piv != p) {
        for (int q = tid; q < w; q += NTC) {
            const int jj = jb + q;
            if (jj >= sb && jj < se) continue;
            const cd t = T[(size_t)p * W + jj];
            T[(size_t)p * W + jj] = T[(size_t)piv * W + jj];
            T[(size_t)piv * W + jj] = t;
        }
        __syncthreads();
    }
    for (int q = tid; q < w; q += NTC) {
        const int jj = jb + q;
        rowp[jj] = (c0 + jj == p) ? inv : cmul(T[(size_t)p * W + jj], inv);
    }
    __syncthreads();
    // elimination mapping: a fixed column and every erows-th row
    const int erows = NTC / w;
    const int ej = tid % w, ei = tid / w;
    if (ei < erows) {
        const int jj = jb + ej;
        if (!(jj >= sb && jj < se)) {
            const cd gg = rowp[jj];
            const bool pcol = (c0 + jj == p);
            for (int i = ei; i < n; i += erows) {
                if (i == p) {
                    T[(size_t)i * W + jj] = gg;
                } else if (pcol) {
                    T[(size_t)i * W + jj] = -cmul(col[i], inv);
                } else {
                    cd v = T[(size_t)i * W + jj];
                    const cd f = col[i];
                    v.re = fma(-f.re, gg.re, v.re);
                    v.re = fma(f.im, gg.im, v.re);
                    v.im = fma(-f.re, gg.im, v.im);
                    v.im = fma(-f.im, gg.re, v.im);
                    T[(size_t)i * W + jj] = v;
                }
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NTC)
    k_newton_cluster(const double2* __restrict__ H, long long h_rhs_stride, int ldh, const int* __restrict__ k_used,
                     const double* __restrict__ beta, double2* __restrict__ coeff, long long coeff_stride,
                     double2* __restrict__ work, int kmax, int kc, int bw, int* __restrict__ iters,
                     int* __restrict__ status, const int* __restrict__ active, int n_fixed) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_pidx[2][kMaxPanel], s_ok[2];
    __shared__ double2 s_pinv[2][kMaxPanel];
    __shared__ int s_piv;
    __shared__ double s_part[2];
    __shared__ double s_red[NTC / 32];
    __shared__ double s_bv[NTC / 32];
    __shared__ int s_bi[NTC / 32];
    __shared__ cd s_inv_l[kMaxPanel];
    __shared__ int s_piv_l[kMaxPanel];
    const int c = (int)cl.block_rank();
    const int ncl = (int)cl.num_blocks();
    const int r = blockIdx.x / ncl;
    const int tid = threadIdx.x;
    if (active != nullptr && active[r] == 0) return;  // uniform over the cluster
    const int n = n_fixed > 0 ? n_fixed : k_used[r];
    // shared-memory layout for matrices of order <= kc (kc <= kmax)
    const int Wmax = (kc + ncl - 1) / ncl;
    cd* T = reinterpret_cast<cd*>(smem_raw);          // [kc][Wmax]
    cd* pub = T + (size_t)kc * Wmax;                  // [2][bw][kc] published panel columns
    cd* colL = pub + 2 * (size_t)bw * kc;             // [bw][kc] local copy of the panel
    cd* rowp = colL + (size_t)bw * kc;                // [Wmax]
    int* perm = reinterpret_cast<int*>(rowp + Wmax);  // [kc]
    int* srcc = perm + kc;                            // [kc]
    double2* cr = coeff + r * coeff_stride;
    if (n <= 0) {
        if (c == 0) {
            for (int i = tid; i < kmax; i += NTC) cr[i] = make_double2(0.0, 0.0);
            if (tid == 0) { iters[r] = 0; status[r] = ST_OK; }
        }
        return;  // uniform over the cluster: n is the same for all its CTAs
    }
    const int W = (n + ncl - 1) / ncl;
    const int c0 = c * W;
    const int w = max(0, min(n, c0 + W) - c0);
    cd* S = reinterpret_cast<cd*>(work) + (size_t)r * 2 * kmax * kmax;  // row-major n x n
    const double2* Hr = H + r * h_rhs_stride;
    for (int idx = tid; idx < n * w; idx += NTC) {
        const int i = idx / w, jj = idx - i * w;
        const double2 h = Hr[i + (long long)(c0 + jj) * ldh];
        S[(size_t)i * n + c0 + jj] = {h.x, h.y};
    }
    int st = ST_NOT_CONVERGED, it_done = 0, remaining = -1;
    for (int it = 1; it <= kMaxIter; ++it) {
        for (int idx = tid; idx < n * w; idx += NTC) {
            const int i = idx / w, jj = idx - i * w;
            T[(size_t)i * W + jj] = S[(size_t)i * n + c0 + jj];
        }
        __syncthreads();
        bool ok = true;
        int panel = 0;
        for (int p0 = 0; p0 < n; ++panel) {
            const int owner = p0 / W;
            const int p1 = min(min(p0 + bw, (owner + 1) * W), n);
            const int cnt = p1 - p0;
            const int buf = panel & 1;
            if (c == owner) {
                // A. the panel's pivots on the panel columns [p0 - c0, p1 - c0)
                if (tid == 0) s_ok[buf] = 1;
                __syncthreads();
                for (int p = p0; p < p1; ++p) {
                    const int jl = p - c0, k = p - p0;
                    double best = -1.0;
                    int bi = p;
                    for (int i = p + tid; i < n; i += NTC) {
                        const cd a = T[(size_t)i * W + jl];
                        const double v = a.re * a.re + a.im * a.im;
                        if (v > best) { best = v; bi = i; }
                    }
                    for (int off = 16; off > 0; off >>= 1) {
                        const double ov = __shfl_xor_sync(0xffffffffu, best, off);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
                    }
                    if ((tid & 31) == 0) { s_bv[tid >> 5] = best; s_bi[tid >> 5] = bi; }
                    __syncthreads();
                    if (tid == 0) {
                        double b = s_bv[0];
                        int ib = s_bi[0];
                        for (int q = 1; q < NTC / 32; ++q)
                            if (s_bv[q] > b || (s_bv[q] == b && s_bi[q] < ib)) { b = s_bv[q]; ib = s_bi[q]; }
                        s_piv = ib;
                        s_pidx[buf][k] = ib;
                        if (!(b > 0.0 && isfinite(b))) s_ok[buf] = 0;
                    }
                    __syncthreads();
                    if (!s_ok[buf]) break;  // uniform over the CTA
                    const int piv = s_piv;
                    cd* pc = pub + ((size_t)buf * bw + k) * kc;
                    for (int i = tid; i < n; i += NTC) {
                        const int si = (i == p) ? piv : (i == piv ? p : i);
                        pc[i] = T[(size_t)si * W + jl];
                    }
                    __syncthreads();
                    if (tid == 0) {  // the pivot's inverse, once per panel column
                        const cd a = pc[p];
                        const double den = a.re * a.re + a.im * a.im;
                        s_pinv[buf][k] = make_double2(a.re / den, -a.im / den);
                    }
                    __syncthreads();
                    const cd inv = {s_pinv[buf][k].x, s_pinv[buf][k].y};
                    gj_apply(T, W, n, c0, p0 - c0, p1 - c0, 0, 0, p, piv, pc, inv, rowp);
                }
            }
            cl.sync();
            // B. the panel's pivots on every other column of this CTA
            if (!*cl.map_shared_rank(&s_ok[buf], owner)) {
                ok = false;
                break;  // uniform over the cluster
            }
            {
                const cd* rpub = cl.map_shared_rank(pub + (size_t)buf * bw * kc, owner);
                for (int idx = tid; idx < cnt * n; idx += NTC) {
                    const int k = idx / n, i = idx - k * n;
                    colL[(size_t)k * kc + i] = rpub[(size_t)k * kc + i];
                }
                if (tid < cnt) {
                    const int* rp = cl.map_shared_rank(&s_pidx[buf][0], owner);
                    const double2* ri = cl.map_shared_rank(&s_pinv[buf][0], owner);
                    s_piv_l[tid] = rp[tid];
                    s_inv_l[tid] = {ri[tid].x, ri[tid].y};
                    perm[p0 + tid] = rp[tid];
                }
            }
            __syncthreads();
            const int sb = (c == owner) ? p0 - c0 : 0, se = (c == owner) ? p1 - c0 : 0;
            for (int k = 0; k < cnt; ++k)
                gj_apply(T, W, n, c0, 0, w, sb, se, p0 + k, s_piv_l[k], colL + (size_t)k * kc, s_inv_l[k], rowp);
            p0 = p1;
        }
        if (!ok) {
            cl.sync();  // the owner's flag was read remotely: no block leaves before all have read it
            st = ST_ESIGN;
            it_done = it;
            break;
        }
        // S^-1 = (Gauss-Jordan result) with the row interchanges undone as
        // column interchanges, last first: column j comes from column srcc[j]
        if (tid == 0) {
            for (int j = 0; j < n; ++j) srcc[j] = j;
            for (int p = n - 1; p >= 0; --p) {
                const int q = perm[p];
                const int t = srcc[p];
                srcc[p] = srcc[q];
                srcc[q] = t;
            }
        }
        cl.sync();  // every block's Gauss-Jordan result is final
        double d2 = 0.0, s2 = 0.0;
        for (int idx = tid; idx < n * w; idx += NTC) {
            const int i = idx / w, jj = idx - i * w;
            const int j = c0 + jj, sj = srcc[j];
            const int ow = sj / W, lj = sj - ow * W;
            const cd b = cl.map_shared_rank(T, ow)[(size_t)i * W + lj];
            const cd a0 = S[(size_t)i * n + j];
            const cd v = {0.5 * (a0.re + b.re), 0.5 * (a0.im + b.im)};
            const double dx = v.re - a0.re, dy = v.im - a0.im;
            d2 += dx * dx + dy * dy;
            s2 += v.re * v.re + v.im * v.im;
            S[(size_t)i * n + j] = v;
        }
        d2 = cl_block_sum(d2, s_red);
        s2 = cl_block_sum(s2, s_red);
        if (tid == 0) { s_part[0] = d2; s_part[1] = s2; }
        cl.sync();  // partials visible; remote reads of T finished
        double D2 = 0.0, S2 = 0.0;
        for (int q = 0; q < ncl; ++q) {
            const double* rp = cl.map_shared_rank(s_part, q);
            D2 += rp[0];
            S2 += rp[1];
        }
        it_done = it;
        const double change = sqrt(D2 / S2);
        cl.sync();  // nobody overwrites s_part or T before all have read them
        if (!isfinite(change)) {
            st = ST_ESIGN;
            break;
        }
        if (remaining < 0 && change <= kSwitchTol) remaining = kExtra;
        if (remaining >= 0) {
            if (remaining == 0) {
                st = ST_OK;
                break;
            }
            --remaining;
        }
    }
    if (c == 0) {
        const double bt = beta[r];
        for (int i = tid; i < kmax; i += NTC) {
            if (i < n && st != ST_ESIGN) {
                const cd sv = S[(size_t)i * n];
                cr[i] = make_double2(bt * sv.re, bt * sv.im);
            } else {
                cr[i] = make_double2(0.0, 0.0);
            }
        }
        if (tid == 0) {
            iters[r] = it_done;
            status[r] = st;
        }
    }
}

// Convergence estimate of the batched form (one block per right-hand side
// that is due): est = ||c_new - c_old|| / ||c_new|| over the coefficient
// vectors of two checks (zero beyond their sizes); below tol the right-hand
// side stops with k_used = n. Otherwise c_new becomes c_old and the next
// check is scheduled: `every` steps on, or with the skip-ahead schedule
// (two one-interval estimates e0 > e1 at j0 < j1) at P = every floor((j1 + n')
// / every) - every, n' = log(tol/e1) / (log(e1/e0)/(j1 - j0)) the steps the
// geometric extrapolation needs to reach tol, P at most cap - every.
__global__ void k_conv_check(const double2* __restrict__ cnew, double2* __restrict__ cold, long long stride, int n,
                             double tol, int* __restrict__ active, int* __restrict__ k_used,
                             double* __restrict__ est, const int* __restrict__ due, CheckState* __restrict__ cs,
                             int every, int cap, int skip) {
    __shared__ double sh[33];
    const int r = blockIdx.x;
    if (due[r] == 0) return;
    double d2 = 0.0, c2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 a = cnew[r * stride + i], b = cold[r * stride + i];
        d2 += (a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y);
        c2 += a.x * a.x + a.y * a.y;
    }
    d2 = blk_sum(d2, sh);
    c2 = blk_sum(c2, sh);  // every read of cold is done: it may be overwritten
    for (int i = threadIdx.x; i < n; i += blockDim.x) cold[r * stride + i] = cnew[r * stride + i];
    if (threadIdx.x == 0) {
        const double e = c2 > 0.0 ? sqrt(d2 / c2) : 0.0;
        est[r] = e;
        if (e < tol) {
            active[r] = 0;
            k_used[r] = n;
            cs[r].next = -1;  // stopped here: cold holds beta sgn(H_n) e_1
            return;
        }
        CheckState s = cs[r];
        int nxt = n + every;
        if (skip && s.jl > 0 && n - s.jl == every) {
            s.j0 = s.j1;
            s.e0 = s.e1;
            s.j1 = n;
            s.e1 = e;
            if (s.j0 > 0 && s.e1 < s.e0) {
                const double steps = log(tol / s.e1) / (log(s.e1 / s.e0) / (double)(s.j1 - s.j0));
                const double t = (double)s.j1 + steps;
                const int pn = t >= (double)cap ? cap - every : every * (int)floor(t / (double)every) - every;
                nxt = max(nxt, pn);
            }
        }
        s.jl = n;
        s.next = nxt;
        cs[r] = s;
    }
}

__global__ void k_check_init(CheckState* __restrict__ cs, int every, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrhs) cs[r] = CheckState{0, 0, 0, every, 0.0, 0.0};
}

__global__ void k_check_due(const int* __restrict__ active, const CheckState* __restrict__ cs, int j,
                            int* __restrict__ due, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrhs) due[r] = (active[r] != 0 && cs[r].next == j) ? 1 : 0;
}

// After the last step: a right-hand side stopped by a check already has its
// coefficients beta sgn(H_k_used) e_1 (in cold): copy them to coeff and
// leave it out of the final sign computation (due = 0); the others are due.
__global__ void k_check_final(const CheckState* __restrict__ cs, const double2* __restrict__ cold,
                              double2* __restrict__ coeff, long long stride, const int* __restrict__ k_used,
                              int* __restrict__ due) {
    const int r = blockIdx.x;
    const bool stopped = cs[r].next == -1;
    if (threadIdx.x == 0) due[r] = stopped ? 0 : 1;
    if (!stopped) return;
    const int n = k_used[r];
    for (int i = threadIdx.x; i < n; i += blockDim.x) coeff[r * stride + i] = cold[r * stride + i];
}

cudaError_t launch_check_final(const CheckState* cs, const void* cold, void* coeff, long long stride,
                               const int* k_used, int* due, int nrhs, cudaStream_t st) {
    k_check_final<<<nrhs, 256, 0, st>>>(cs, (const double2*)cold, (double2*)coeff, stride, k_used, due);
    return cudaGetLastError();
}

cudaError_t launch_check_init(CheckState* cs, int every, int nrhs, cudaStream_t st) {
    k_check_init<<<(nrhs + 127) / 128, 128, 0, st>>>(cs, every, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_check_due(const int* active, const CheckState* cs, int j, int* due, int nrhs, cudaStream_t st) {
    k_check_due<<<(nrhs + 127) / 128, 128, 0, st>>>(active, cs, j, due, nrhs);
    return cudaGetLastError();
}

cudaError_t launch_conv_check(const void* cnew, void* cold, long long stride, int n, double tol, int* active,
                              int* k_used, double* est, const int* due, CheckState* cs, int every, int cap,
                              bool skip, int nrhs, cudaStream_t st) {
    k_conv_check<<<nrhs, 256, 0, st>>>((const double2*)cnew, (double2*)cold, stride, n, tol, active, k_used, est,
                                       due, cs, every, cap, skip ? 1 : 0);
    return cudaGetLastError();
}

// Harmonic variant (the see-saw-free form cited in Sec. 4): H_k is replaced
// by H^_k = H_k + |h_(k+1,k)|^2 f e_k^T with f = H_k^-H e_k, whose
// eigenvalues are the harmonic Ritz values. One block per right-hand side.
// f from a Givens QR of the Hessenberg H_k: rotations G_j (rows j, j+1)
// with G_(k-2) ... G_0 H_k = R give H_k = Q R, Q = G_0^H ... G_(k-2)^H, and
// H_k^H f = e_k is R^H (Q^H f) = e_k, so f = Q e_k / conj(R_kk). The copy of
// H_k and the rotations live in `work` (2 kmax^2 complex128 per right-hand
// side, the Newton work space, free before the Newton kernel runs).
// Right-hand sides after a breakdown (h_(k+1,k) = 0) keep H_k.
__global__ void __launch_bounds__(256) k_harmonic(double2* __restrict__ H, long long h_rhs_stride, int ldh,
                                                  const int* __restrict__ k_used, double2* __restrict__ work,
                                                  int kmax) {
    __shared__ double2 s_rot[2];
    const int r = blockIdx.x, tid = threadIdx.x;
    const int n = k_used[r];
    double2* Hr = H + r * h_rhs_stride;
    if (n < 1) return;
    const double2 sub = Hr[n + (long long)(n - 1) * ldh];
    const double h2 = sub.x * sub.x + sub.y * sub.y;
    if (!(h2 > 0.0)) return;
    cd* W = reinterpret_cast<cd*>(work) + (size_t)r * 2 * kmax * kmax;  // row-major n x n
    cd* rot = W + (size_t)kmax * kmax;                                // (a/rho, b/rho) per step
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx - i * n;
        const double2 h = (i <= j + 1) ? Hr[i + (long long)j * ldh] : make_double2(0.0, 0.0);
        W[idx] = {h.x, h.y};
    }
    __syncthreads();
    for (int j = 0; j + 1 < n; ++j) {
        if (tid == 0) {
            const cd a = W[(size_t)j * n + j], b = W[(size_t)(j + 1) * n + j];
            const double rho = sqrt(a.re * a.re + a.im * a.im + b.re * b.re + b.im * b.im);
            if (rho > 0.0 && isfinite(rho)) {
                s_rot[0] = make_double2(a.re / rho, a.im / rho);
                s_rot[1] = make_double2(b.re / rho, b.im / rho);
            } else {
                s_rot[0] = make_double2(1.0, 0.0);
                s_rot[1] = make_double2(0.0, 0.0);
            }
            rot[2 * j] = {s_rot[0].x, s_rot[0].y};
            rot[2 * j + 1] = {s_rot[1].x, s_rot[1].y};
        }
        __syncthreads();
        // G = [[conj(a), conj(b)], [-b, a]] / rho on rows j, j+1
        const cd ca = {s_rot[0].x, s_rot[0].y}, cb = {s_rot[1].x, s_rot[1].y};
        for (int l = j + tid; l < n; l += blockDim.x) {
            const cd w1 = W[(size_t)j * n + l], w2 = W[(size_t)(j + 1) * n + l];
            W[(size_t)j * n + l] = cmulc(ca, w1) + cmulc(cb, w2);
            W[(size_t)(j + 1) * n + l] = cmul(ca, w2) - cmul(cb, w1);
        }
        __syncthreads();
    }
    if (tid == 0) {
        // v = Q e_n = G_0^H ... G_(n-2)^H e_n; G^H = [[a, -conj(b)], [b, conj(a)]] / rho
        cd* v = W;  // row 0 of W is no longer needed: reuse it for v
        const cd rnn = W[(size_t)(n - 1) * n + (n - 1)];
        for (int i = 0; i < n; ++i) v[i] = {0.0, 0.0};
        v[n - 1] = {1.0, 0.0};
        for (int j = n - 2; j >= 0; --j) {
            const cd a = rot[2 * j], b = rot[2 * j + 1];
            const cd v1 = v[j], v2 = v[j + 1];
            v[j] = cmul(a, v1) - cmulc(b, v2);
            v[j + 1] = cmul(b, v1) + cmulc(a, v2);
        }
        // f = v / conj(rnn); H[:, n-1] += |h|^2 f
        const double den = rnn.re * rnn.re + rnn.im * rnn.im;
        if (den > 0.0 && isfinite(den)) {
            const cd inv_conj = {rnn.re / den, rnn.im / den};  // 1 / conj(rnn) = rnn / |rnn|^2
            for (int i = 0; i < n; ++i) {
                const cd f = cmul(v[i], inv_conj);
                double2 h = Hr[i + (long long)(n - 1) * ldh];
                h.x += h2 * f.re;
                h.y += h2 * f.im;
                Hr[i + (long long)(n - 1) * ldh] = h;
            }
        }
    }
    // a singular H_k (R_kk = 0) is left unmodified: the Newton iteration on
    // it then reports OVS_ESIGN
}

cudaError_t launch_harmonic(void* H, long long h_rhs_stride, int ldh, const int* k_used, void* work, int kmax,
                            int nrhs, cudaStream_t st) {
    k_harmonic<<<nrhs, 256, 0, st>>>((double2*)H, h_rhs_stride, ldh, k_used, (double2*)work, kmax);
    return cudaGetLastError();
}

static size_t cluster_smem(int kmax, int ncl, int bw) {
    const int Wmax = (kmax + ncl - 1) / ncl;
    return ((size_t)kmax * Wmax + 3 * (size_t)bw * kmax + Wmax) * sizeof(cd) + 2 * (size_t)kmax * sizeof(int);
}

constexpr size_t kClusterSmemMax = 220 * 1024;

// Widest panel (8, 4, 2 or 1 columns) whose buffers fit next to the blocks
// of a cluster of ncl CTAs; 0 if not even one column fits.
static int panel_width(int kmax, int ncl) {
    for (int bw = kMaxPanel; bw >= 1; bw /= 2)
        if (cluster_smem(kmax, ncl, bw) <= kClusterSmemMax) return bw;
    return 0;
}

// Cluster size for nrhs matrices of order <= kmax: the candidate with the
// fewest waves per SM of a cluster (waves / ncl, the FP64 work per SM being
// proportional to 1/ncl), 0 if none fits. Clusters of one block per SM are
// placed within a GPC, so how many are resident at once depends on the size
// and is asked of the runtime (cached per size and shared-memory need).
static int pick_cluster(int kmax, int nrhs) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, int> resident;  // (device, size, smem) -> clusters
    if (ensure_dyn_smem((const void*)k_newton_cluster, kClusterSmemMax) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    int best = 0;
    double best_cost = 0.0;
    for (int ncl : kClusterSizes) {
        const int bw = panel_width(kmax, ncl);
        if (bw == 0) continue;
        const size_t need = cluster_smem(kmax, ncl, bw);
        auto key = std::make_tuple(dev, ncl, need);
        auto it = resident.find(key);
        if (it == resident.end()) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = ncl;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(ncl);
            cfg.blockDim = dim3(NTC);
            cfg.dynamicSmemBytes = need;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_newton_cluster, &cfg) != cudaSuccess) {
                cudaGetLastError();
                n = 0;
            }
            it = resident.emplace(key, n).first;
        }
        if (it->second < 1) continue;
        const int waves = (nrhs + it->second - 1) / it->second;
        const double cost = (double)waves / ncl;
        if (best == 0 || cost < best_cost - 1e-12) {
            best = ncl;
            best_cost = cost;
        }
    }
    return best;
}

cudaError_t launch_newton(const void* H, long long h_rhs_stride, int ldh, const int* k_used, const double* beta,
                          void* coeff, long long coeff_stride, void* work, int kmax, int nrhs, int* iters,
                          int* status, cudaStream_t st, const int* active, int n_fixed, int k_bound) {
    // matrices of a known order (the convergence checks), or of orders
    // bounded by the call's Krylov dimension, need shared memory for that
    // order only, so they can use the cluster form below kmax (the work
    // space may have been sized by an earlier call with a larger k)
    int kc = kmax;
    if (n_fixed > 0 && n_fixed < kmax)
        kc = n_fixed;
    else if (n_fixed <= 0 && k_bound > 0 && k_bound < kmax)
        kc = k_bound;
    const int ncl = pick_cluster(kc, nrhs);
    if (ncl > 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = ncl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(nrhs * ncl);
        cfg.blockDim = dim3(NTC);
        const int bw = panel_width(kc, ncl);
        cfg.dynamicSmemBytes = cluster_smem(kc, ncl, bw);
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_newton_cluster, (const double2*)H, h_rhs_stride, ldh, k_used, beta,
                                  (double2*)coeff, coeff_stride, (double2*)work, kmax, kc, bw, iters, status, active,
                                  n_fixed);
    }
    const size_t smem = (size_t)kmax * 2 * sizeof(cd) + (size_t)kmax * sizeof(int);
    const cudaError_t e = ensure_dyn_smem((const void*)k_newton, 200 * 1024);
    if (e != cudaSuccess) return e;
    k_newton<<<nrhs, NT, smem, st>>>((const double2*)H, h_rhs_stride, ldh, k_used, beta, (double2*)coeff,
                                     coeff_stride, (double2*)work, kmax, iters, status, active, n_fixed);
    return cudaGetLastError();
}

}  // namespace ovs
