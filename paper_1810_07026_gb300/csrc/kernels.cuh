// Compute kernels of one step (templated on the arithmetic type R).
//
//   short_list  : exact REBO neighbours (r < Dmax_ij) from the intermediate
//                 list, w and dw/dr, N^C, N^H per atom, the i<j bond list
//                 (Sec. 4.1: rebuilt every step from a list with a skin)
//   rebo        : one thread per bond: b_ij forward + reverse, E = f_R + b f_A (Alg. 1)
//   torsion     : one thread per C-C bond (Alg. 2)
//   path_map    : one thread per atom: connectivity map over <= 3 bonds, the
//                 reverse of the per-pair C_ij search (Sec. 4.3)
//   lj          : one warp per atom i, lanes over its half list: cut-off test,
//                 C_ij lookup, V^LJ, forces; pairs with S_r != 0 are queued
//                 for b* (the deferred batch of Sec. 4.3)
//   bstar       : one thread per queued pair: b*, S_b, forces (Alg. 3)
#pragma once

#include "internal.h"

namespace airebo {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide accumulation of an energy and the virial into global sums
template <int NT>
__device__ void block_accumulate(double e, const double* W, bool virial, double* accE, double* accW) {
    __shared__ double red[NT / 32][7];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    e = warp_sum(e);
    double w[6];
    for (int k = 0; k < 6; k++) w[k] = virial ? warp_sum(W[k]) : 0.0;
    if (lane == 0) {
        red[wid][0] = e;
        for (int k = 0; k < 6; k++) red[wid][k + 1] = w[k];
    }
    __syncthreads();
    if (threadIdx.x < 7 && (threadIdx.x == 0 || virial)) {
        double s = 0;
        for (int q = 0; q < NT / 32; q++) s += red[q][threadIdx.x];
        if (threadIdx.x == 0) atomicAdd(accE, s);
        else atomicAdd(accW + threadIdx.x - 1, s);
    }
}

__device__ __forceinline__ void load_disp(const double* pos, int n, const double* L, int i, int j, int img,
                                          double& dx, double& dy, double& dz) {
    dx = pos[j] + img_x(img) * L[0] - pos[i];
    dy = pos[n + j] + img_y(img) * L[1] - pos[n + i];
    dz = pos[2 * n + j] + img_z(img) * L[2] - pos[2 * n + i];
}

// ------------------------------------------------------------------ short list
template <class R>
__global__ void __launch_bounds__(128) k_short_list(StepArgs<R> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const DevParams<R>& P = *a.P;
    int n = a.n;
    double xi = a.pos[i], yi = a.pos[n + i], zi = a.pos[2 * n + i];
    if (!isfinite(xi) || !isfinite(yi) || !isfinite(zi)) atomicMax(a.err + ERR_NONFINITE, 1);
    int ti = a.G.type[i];
    int cnt = 0;
    R nC = 0, nH = 0;
    int ne = a.im_cnt[i];
    const int2* row = a.im + (size_t)i * a.im_cap;
    for (int e = 0; e < ne; e++) {
        int2 ent = row[e];
        int j = ent.x, img = ent.y;
        double dx = a.pos[j] + img_x(img) * a.L[0] - xi;
        double dy = a.pos[n + j] + img_y(img) * a.L[1] - yi;
        double dz = a.pos[2 * n + j] + img_z(img) * a.L[2] - zi;
        double r2 = dx * dx + dy * dy + dz * dz;
        int tj = a.G.type[j];
        int p = pidx(ti, tj);
        double dmax = (double)P.Dmax[p];
        if (!(r2 < dmax * dmax)) continue;
        double r = sqrt(r2);
        R dw;
        R w = wfun<R>(P, p, (R)r, dw);
        if (cnt < MAXN) {
            int q = i * MAXN + cnt;
            a.g_nj[q] = j; a.g_nimg[q] = img;
            a.g_dx[q] = (R)dx; a.g_dy[q] = (R)dy; a.g_dz[q] = (R)dz;
            a.g_r[q] = (R)r; a.g_w[q] = w; a.g_dw[q] = dw;
            if (j > i) {
                int b = atomicAdd(a.nbonds, 1);
                if (b < a.bond_cap) a.bonds[b] = make_int2(i, cnt);
            }
        }
        cnt++;
        if (tj == 0) nC += w; else nH += w;
    }
    if (cnt > MAXN) atomicMax(a.err + ERR_SHORT, cnt);
    a.g_cnt[i] = cnt < MAXN ? cnt : MAXN;
    a.g_nC[i] = nC;
    a.g_nH[i] = nH;
}

// ------------------------------------------------------------------ REBO bonds
template <class R>
__global__ void __launch_bounds__(128) k_rebo(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, a.virial, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    int nb = *a.nbonds;
    if (nb > a.bond_cap) nb = a.bond_cap;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int2 bd = a.bonds[b];
        E += rebo_bond<R>(P, a.G, bd.x, bd.y, sink);
    }
    block_accumulate<128>(E, sink.W, a.virial, a.acc + 0, a.acc + 3);
}

// ------------------------------------------------------------------ torsion
template <class R>
__global__ void __launch_bounds__(128) k_torsion(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, a.virial, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    int nb = *a.nbonds;
    if (nb > a.bond_cap) nb = a.bond_cap;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int2 bd = a.bonds[b];
        int j = a.G.nj[bd.x * MAXN + bd.y];
        if (a.G.type[bd.x] != 0 || a.G.type[j] != 0) continue;
        E += torsion_bond<R>(P, a.G, bd.x, bd.y, sink);
    }
    block_accumulate<128>(E, sink.W, a.virial, a.acc + 2, a.acc + 3);
}

// ------------------------------------------------------------------ connectivity map
template <class R>
__global__ void __launch_bounds__(128) k_path_map(StepArgs<R> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    PathMap<R> M = a.M;
    int ov = build_path_map<R>(a.G, M, i);
    if (ov) atomicMax(a.err + ERR_MAP, M.cnt[i] + ov);
}

template <class R>
__device__ __forceinline__ int map_find(const PathMap<R>& M, int i, long long key) {
    int c = M.cnt[i];
    const long long* k = M.key + (size_t)i * M.cap;
    for (int e = 0; e < c; e++)
        if (k[e] == key) return e;
    return -1;
}

// ------------------------------------------------------------------ LJ
template <class R>
__global__ void __launch_bounds__(256) k_lj(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    int lane = threadIdx.x & 31;
    int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Sink sink{a.f, a.n, a.virial, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    unsigned evaluated = 0;
    if (i < a.n) {
        int n = a.n;
        double xi = a.pos[i], yi = a.pos[n + i], zi = a.pos[2 * n + i];
        int ti = a.G.type[i];
        double fix = 0, fiy = 0, fiz = 0;
        int ne = a.lj_cnt[i];
        const int2* row = a.lj + (size_t)i * a.lj_cap;
        for (int e = lane; e < ne; e += 32) {
            int2 ent = row[e];
            int j = ent.x, img = ent.y;
            // displacement in FP64 (minimum-image arithmetic stays double)
            double dx = a.pos[j] + img_x(img) * a.L[0] - xi;
            double dy = a.pos[n + j] + img_y(img) * a.L[1] - yi;
            double dz = a.pos[2 * n + j] + img_z(img) * a.L[2] - zi;
            R rx = (R)dx, ry = (R)dy, rz = (R)dz;
            R r2 = rx * rx + ry * ry + rz * rz;
            int p = pidx(ti, a.G.type[j]);
            if (!(r2 < P.rc2[p])) continue;
            evaluated++;
            R C = R(1);
            int mi = -1, code = -1;
            if (r2 < P.rpath2) {
                mi = map_find<R>(a.M, i, map_key(j, img));
                if (mi >= 0) {
                    R wm = a.M.wt[(size_t)i * a.M.cap + mi];
                    if (wm >= R(1)) continue;
                    C = R(1) - wm;
                    code = a.M.path[(size_t)i * a.M.cap + mi];
                }
            }
            R rr = sqrt_(r2);
            if (rr < P.Srhi[p]) {
                int q = atomicAdd(a.nbq, 1);
                if (q < a.bq_cap) a.bq[q] = make_int4(i, e, mi, 0);
                continue;
            }
            R inv_r = R(1) / rr;
            R dV;
            R V = vlj<R>(P, p, rr, inv_r * inv_r, dV);
            E += (double)(C * V);
            double c = (double)(C * dV * inv_r);
            double gx = c * dx, gy = c * dy, gz = c * dz;
            sink.half(j, dx, dy, dz, gx, gy, gz, fix, fiy, fiz);
            if (code >= 0) path_forces<R>(a.G, i, code, -V, sink, fix, fiy, fiz);
        }
        fix = warp_sum(fix); fiy = warp_sum(fiy); fiz = warp_sum(fiz);
        if (lane == 0) {
            atomicAdd(a.f + i, fix); atomicAdd(a.f + n + i, fiy); atomicAdd(a.f + 2 * n + i, fiz);
        }
    }
    unsigned ev = __reduce_add_sync(0xffffffffu, evaluated);
    if (lane == 0 && ev) atomicAdd(a.counters + CNT_LJ, (unsigned long long)ev);
    block_accumulate<256>(E, sink.W, a.virial, a.acc + 1, a.acc + 3);
}

// ------------------------------------------------------------------ b* pairs
template <class R>
__global__ void __launch_bounds__(128) k_bstar(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, a.virial, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    unsigned dsb = 0;
    int nq = *a.nbq;
    if (nq > a.bq_cap) nq = a.bq_cap;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += gridDim.x * blockDim.x) {
        int4 q = a.bq[t];
        int i = q.x;
        int2 ent = a.lj[(size_t)i * a.lj_cap + q.y];
        int j = ent.x;
        double dx, dy, dz;
        load_disp(a.pos, a.n, a.L, i, j, ent.y, dx, dy, dz);
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        R C = R(1);
        int code = -1;
        if (q.z >= 0) {
            C = R(1) - a.M.wt[(size_t)i * a.M.cap + q.z];
            code = a.M.path[(size_t)i * a.M.cap + q.z];
        }
        E += bstar_pair<R>(P, a.G, i, j, (R)dx, (R)dy, (R)dz, (R)r, C, code, sink, &dsb);
    }
    unsigned s = __reduce_add_sync(0xffffffffu, dsb);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(a.counters + CNT_DSB, (unsigned long long)s);
    block_accumulate<128>(E, sink.W, a.virial, a.acc + 1, a.acc + 3);
}

template <class R>
__global__ void k_finish_counters(StepArgs<R> a) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        a.counters[CNT_BONDS] = (unsigned long long)*a.nbonds;
        a.counters[CNT_BSTAR] = (unsigned long long)*a.nbq;
    }
}

template <class R>
void launch_compute_impl(const StepArgs<R>& a, cudaStream_t s, int num_sms, cudaEvent_t* ev) {
    if (a.n == 0) return;
    int n = a.n;
    auto mark = [&](int k) { if (ev) cudaEventRecord(ev[k], s); };
    int grid_bonds = num_sms * 8;
    mark(0);
    k_short_list<R><<<(n + 127) / 128, 128, 0, s>>>(a);
    mark(1);
    if (a.rebo) k_rebo<R><<<grid_bonds, 128, 0, s>>>(a);
    mark(2);
    if (a.torsion) k_torsion<R><<<grid_bonds, 128, 0, s>>>(a);
    mark(3);
    if (a.lj_on) k_path_map<R><<<(n + 127) / 128, 128, 0, s>>>(a);
    mark(4);
    if (a.lj_on) k_lj<R><<<(n + 7) / 8, 256, 0, s>>>(a);
    mark(5);
    if (a.lj_on) k_bstar<R><<<grid_bonds, 128, 0, s>>>(a);
    mark(6);
    k_finish_counters<R><<<1, 32, 0, s>>>(a);
}

}  // namespace airebo
