// Compute kernels of one step (templated on the arithmetic type R).
//
//   posf        : one thread per atom: FP32 (or split hi + lo) positions for
//                 the FP32 pre-tests
//   short_list  : exact REBO neighbours (r < Dmax_ij) from the intermediate
//                 list, w and dw/dr, N^C, N^H per atom, the i<j bond list
//                 (Sec. 4.1: rebuilt every step from a list with a skin)
//   rebo        : one thread per bond: b_ij forward + reverse, E = f_R + b f_A (Alg. 1)
//   torsion     : one thread per C-C bond (Alg. 2); torsion_dd the same in
//                 double-float for AIREBO_DF64
//   path_map    : one thread per atom: connectivity map over <= 3 bonds, the
//                 reverse of the per-pair C_ij search (Sec. 4.3)
//   lj          : persistent warps over chunks of atoms, lanes over an atom's
//                 half list: cut-off test, C_ij lookup, then the live pairs
//                 compacted into batches of 32 for V^LJ and forces; pairs
//                 with S_r != 0 are queued for b* (the deferred batch of Sec. 4.3)
//   bstar       : one thread per queued pair: b*, S_b, forces (Alg. 3), in
//                 two passes (pairs whose S_b is exactly 0 or 1, then the rest)
//
// Kernels with an EXTRA template flag have an instance without virial and
// parameter-gradient accumulators, used whenever neither is asked for; the
// LJ and b* kernels have a MODE instead (0 plain, 1 virial or parameter
// gradient, 2 also the parameter derivatives of the forces).
#pragma once

#include <type_traits>

#include "internal.h"
#include "ff.cuh"

namespace airebo {

// hi/lo split of a double on the 2^-12 grid
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
    double q = rint(v * 4096.0) * (1.0 / 4096.0);
    h = (float)q;
    l = (float)(v - q);
}


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

// block-wide sum of the parameter-gradient accumulators into pg[6]
template <int NT>
__device__ void block_accumulate_g(const double* G, double* pg) {
    __shared__ double red[NT / 32][6];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double g[6];
    for (int k = 0; k < 6; k++) g[k] = warp_sum(G[k]);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < 6; k++) red[wid][k] = g[k];
    __syncthreads();
    if (threadIdx.x < 6) {
        double s = 0;
        for (int q = 0; q < NT / 32; q++) s += red[q][threadIdx.x];
        atomicAdd(pg + threadIdx.x, s);
    }
}

// the periodic box of atom i: the single system's, or its system's
template <class R>
__device__ __forceinline__ const double* box_of(const StepArgs<R>& a, int i) {
    return a.sys ? a.Lsys + 3 * a.sys[i] : a.L;
}

// Per-atom energies: each bond, torsion or pair term is split evenly between
// the two atoms that define it (i and j of the bond or pair), so that the
// per-atom energies do not depend on the atom numbering and sum to the total.
__device__ __forceinline__ void eatom_pair(double* eatom, int i, int j, double e) {
    atomicAdd(eatom + i, 0.5 * e);
    atomicAdd(eatom + j, 0.5 * e);
}

__device__ __forceinline__ void load_disp(const double* pos, int n, const double* L, int i, int j, int img,
                                          double& dx, double& dy, double& dz) {
    if (img == 0) {
        dx = pos[j] - pos[i]; dy = pos[n + j] - pos[n + i]; dz = pos[2 * n + j] - pos[2 * n + i];
    } else {
        dx = pos[j] + img_x(img) * L[0] - pos[i];
        dy = pos[n + j] + img_y(img) * L[1] - pos[n + i];
        dz = pos[2 * n + j] + img_z(img) * L[2] - pos[2 * n + i];
    }
}

// ------------------------------------------------------------------ FP32 positions
// FP32 position and species of every atom for the FP32 pre-tests of the
// short-list and LJ kernels; with split positions (fixed-point LJ sums) the
// FP32 position is the hi part, on the 2^-12 A grid, and pq_lo holds the rest.
template <class R>
__global__ void __launch_bounds__(128) k_posf(StepArgs<R> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int n = a.n;
    double xi = a.pos[i], yi = a.pos[n + i], zi = a.pos[2 * n + i];
    if (!isfinite(xi) || !isfinite(yi) || !isfinite(zi)) atomicOr(a.err + ERR_NONFINITE, NONFINITE_POS);
    if (a.fix) {
        if (!(fabs(xi) < 2000.0 && fabs(yi) < 2000.0 && fabs(zi) < 2000.0)) atomicOr(a.err + ERR_DF, DF_RANGE);
        float4 h, l;
        df_split(xi, h.x, l.x); df_split(yi, h.y, l.y); df_split(zi, h.z, l.z);
        h.w = __int_as_float((int)a.G.type[i]);
        l.w = 0.0f;
        a.posf[i] = h;
        a.pq_lo[i] = l;
    } else {
        a.posf[i] = make_float4((float)xi, (float)yi, (float)zi, __int_as_float((int)a.G.type[i]));
    }
}

// ------------------------------------------------------------------ short list
// Most entries of the intermediate list lie beyond D_max (in hydrocarbons
// about 12 of 14): an FP32 distance on the FP32 positions rules those out
// without FP64 instructions.  Per component the FP32 displacement f differs
// from the FP64 one d by at most e = 2^-22 (2 |x_i| + 4 |S| L + 8) (the
// roundings of x_i, x_j, S L and of the FP32 additions, with |x_j| <= |x_i| +
// |d| + |S| L and a factor of about 2 to spare), plus 2^-11 for split
// positions (hi parts on the 2^-12 grid).  Then |r2f - r2| <= e (2 sum |f_c|
// + 3 e) plus the rounding of r2f, and an entry with r2f beyond D_max^2 by
// more than that is beyond D_max in FP64 too.  The others take the exact FP64
// test.
template <class R>
__global__ void __launch_bounds__(128) k_short_list(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    // D_max^2 by species pair: in FP32 with the pre-test's factor, and in FP64
    __shared__ float dm2f[3];
    __shared__ double dm2[3];
    // per warp: the entries that passed the FP32 pre-test, as (owner lane,
    // entry), evaluated in FP64 32 at a time; and each lane's slot count
    __shared__ int q_e[4][64];
    __shared__ int q_l[4][64];
    __shared__ int s_cnt[4][32];
    if (threadIdx.x < 3) {
        double d = (double)P.Dmax[threadIdx.x];
        float df = (float)d;
        dm2f[threadIdx.x] = df * df * 1.000001f;
        dm2[threadIdx.x] = d * d;
    }
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    s_cnt[wib][lane] = 0;
    __syncthreads();
    int n = a.n;
    int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31);     // the warp's first atom
    int i = i0 + lane;
    bool act = i < n;
    int ne = 0;
    float4 pfi = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int ti = 0;
    if (act) {
        ne = a.im_cnt[i];
        pfi = a.posf[i];
        ti = a.G.type[i];
    }
    float err0 = 2.3841858e-7f * (2.0f * fmaxf(fabsf(pfi.x), fmaxf(fabsf(pfi.y), fabsf(pfi.z))) + 8.0f) +
                 (a.fix ? 4.8828125e-4f : 0.0f);
    const int2* row = a.im + (size_t)(act ? i : 0) * a.im_cap;
    const double* L = box_of(a, act ? i : 0);
    float Lf[3] = {(float)L[0], (float)L[1], (float)L[2]};
    float Lmax = fmaxf(Lf[0], fmaxf(Lf[1], Lf[2]));
    unsigned lt = (1u << lane) - 1u;
    int qn = 0;
    // the FP64 test and the slot of queued entry k (this lane's), for the whole warp
    auto batch = [&](int k) {
        bool have = lane < k;
        int ol = have ? q_l[wib][lane] : 0, e = have ? q_e[wib][lane] : 0;
        int io = i0 + ol;
        bool pass = false;
        int j = 0, img = 0, to = 0, tj = 0, p = 0;
        double dx = 0, dy = 0, dz = 0, r2 = 1;
        if (have) {
            int2 ent = a.im[(size_t)io * a.im_cap + e];
            j = ent.x; img = ent.y;
            to = a.G.type[io]; tj = a.G.type[j];
            p = pidx(to, tj);
            if (img == 0) {               // most entries: no image, three FP64 operations
                dx = a.pos[j] - a.pos[io]; dy = a.pos[n + j] - a.pos[n + io]; dz = a.pos[2 * n + j] - a.pos[2 * n + io];
            } else {
                const double* Lo = box_of(a, io);
                dx = a.pos[j] + img_x(img) * Lo[0] - a.pos[io];
                dy = a.pos[n + j] + img_y(img) * Lo[1] - a.pos[n + io];
                dz = a.pos[2 * n + j] + img_z(img) * Lo[2] - a.pos[2 * n + io];
            }
            r2 = dx * dx + dy * dy + dz * dz;
            pass = lt_nonneg(r2, dm2[p]);            // r2 >= 0; a NaN is not below
            // two atoms at (nearly) one point: every term diverges there
            if (pass && !(r2 > 1e-12)) { atomicOr(a.err + ERR_NONFINITE, NONFINITE_OVERLAP); pass = false; }
        }
        // slots in entry order: the entries of one atom sit in the queue in
        // the order of its row, and take consecutive slots after its count
        unsigned mp = __ballot_sync(0xffffffffu, pass);
        unsigned peers = __match_any_sync(0xffffffffu, pass ? ol : 32 + lane) & mp;
        int rank = __popc(peers & lt);
        int slot = pass ? s_cnt[wib][ol] + rank : 0;
        __syncwarp();
        if (pass && rank == __popc(peers) - 1) s_cnt[wib][ol] = slot + 1;
        __syncwarp();
        if (pass && slot < a.G.stride) {
            double ir = rsqrt_(r2);
            double r = r2 * ir;
            R dw, omw;
            R w = wfun_c<R>(P, p, (R)r, dw, omw);
            int q = io * a.G.stride + slot;
            a.g_nj[q] = j; a.g_nimg[q] = img;
            a.g_dx[q] = (R)dx; a.g_dy[q] = (R)dy; a.g_dz[q] = (R)dz;
            a.g_r[q] = (R)r; a.g_ir[q] = (R)ir; a.g_w[q] = w; a.g_dw[q] = dw; a.g_omw[q] = omw;
            if (a.screen) {
                a.s_dx[q] = (float)dx; a.s_dy[q] = (float)dy; a.s_dz[q] = (float)dz;
                a.s_r[q] = (float)r; a.s_ir[q] = (float)ir; a.s_w[q] = ef_mark_inexact((double)w);
            }
            // each bond once: i < j between like species, from the carbon for C-H,
            // so that the threads of a warp run the same code (species batches, Sec. 4.2)
            bool mine = (to == tj) ? (j > io) : (to == 0);
            if (mine) {
                if (to == 0 && tj == 0) {
                    int c = atomicAdd(a.nccbonds, 1);
                    if (c < a.bond_cap) a.ccbonds[c] = make_int2(io, slot);
                } else if (to == 1 && tj == 1) {   // H-H bonds from the far end of the same array
                    int b = atomicAdd(a.nhhbonds, 1);
                    if (b < a.bond_cap) a.bonds[a.bond_cap - 1 - b] = make_int2(io, slot);
                } else {
                    int b = atomicAdd(a.nbonds, 1);
                    if (b < a.bond_cap) a.bonds[b] = make_int2(io, slot);
                }
            }
        }
    };
    int nmax = __reduce_max_sync(0xffffffffu, ne);
    for (int e = 0; e < nmax; e++) {
        bool keep = false;
        if (e < ne) {
            int2 ent = row[e];
            int j = ent.x, img = ent.y;
            float4 pj = a.posf[j];
            int p = pidx(ti, __float_as_int(pj.w));
            float fx = pj.x - pfi.x, fy = pj.y - pfi.y, fz = pj.z - pfi.z;
            float err = err0;
            if (img != 0) {
                int sx = img_x(img), sy = img_y(img), sz = img_z(img);
                fx += (float)sx * Lf[0]; fy += (float)sy * Lf[1]; fz += (float)sz * Lf[2];
                err += 9.5367432e-7f * (float)max(abs(sx), max(abs(sy), abs(sz))) * Lmax;    // 2^-22 4 |S| L
            }
            // |r2f - r2| <= sum_c |f_c - d_c| (2 |f_c| + |f_c - d_c|) + rounding
            float r2f = fx * fx + fy * fy + fz * fz;
            float band = err * (2.0f * (fabsf(fx) + fabsf(fy) + fabsf(fz)) + 3.0f * err) + 1e-6f * r2f;
            keep = !(r2f > dm2f[p] + band);
        }
        unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int s = qn + __popc(m & lt);
            q_l[wib][s] = lane; q_e[wib][s] = e;
        }
        qn += __popc(m);
        __syncwarp();
        if (qn >= 32) {
            batch(32);
            __syncwarp();
            if (lane < qn - 32) {
                q_l[wib][lane] = q_l[wib][32 + lane]; q_e[wib][lane] = q_e[wib][32 + lane];
            }
            qn -= 32;
            __syncwarp();
        }
    }
    if (qn > 0) batch(qn);
    __syncwarp();
    if (!act) return;
    int cnt = s_cnt[wib][lane];
    int c = cnt < a.G.stride ? cnt : a.G.stride;
    if (cnt > a.G.stride) atomicMax(a.err + ERR_SHORT, cnt);
    // the coordinations, summed over the slots in row order
    R nC = 0, nH = 0;
    for (int s = 0; s < c; s++) {
        int q = i * a.G.stride + s;
        R w = a.g_w[q];
        if (a.G.type[a.g_nj[q]] == 0) nC += w; else nH += w;
    }
    a.g_cnt[i] = c;
    a.g_nC[i] = nC;
    a.g_nH[i] = nH;
    if (a.screen) {
        a.s_nC[i] = ef_mark_inexact((double)nC);
        a.s_nH[i] = ef_mark_inexact((double)nH);
    }
}

// Groups the items of one pass of a block of NT threads (one item per
// thread, or none) by a small key, so that the threads of a warp take items
// with equal keys -- for the bond-order kernels bond_key, i.e. equal loop trip
// counts and spline paths: a counting sort in shared memory.
// key in [0, 64) for an item, -1 for none; returns the item this thread
// takes, or -1.  Every thread of the block calls it.
template <int NT>
__device__ int block_group(int key, int item, int* s_cnt /* 65 */, int* s_item /* NT */) {
    int t = threadIdx.x;
    for (int k = t; k <= 64; k += NT) s_cnt[k] = 0;
    __syncthreads();
    int kk = key < 0 ? 64 : key;
    int rank = atomicAdd(s_cnt + kk, 1);
    __syncthreads();
    if (t < 32) {                     // exclusive scan of the 64 key counts (the empty bucket last)
        int v0 = s_cnt[2 * t], v1 = s_cnt[2 * t + 1], x = v0 + v1;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (t >= o) x += y;
        }
        int ex = x - v0 - v1;
        __syncwarp();
        s_cnt[2 * t] = ex;
        s_cnt[2 * t + 1] = ex + v0;
        if (t == 31) s_cnt[64] = x;
    }
    __syncthreads();
    s_item[s_cnt[kk] + rank] = key < 0 ? -1 : item;
    __syncthreads();
    int r = s_item[t];
    __syncthreads();                  // the arrays are rewritten by the next pass
    return r;
}
// the grouping key of a pair of atoms for their bond order: the sum of their
// neighbour counts (loop trip counts) and whether each coordination is an
// integer (the spline knot paths)
template <class R> __device__ __forceinline__ int bond_key(const Graph<R>& G, int i, int j) {
    R Ni = G.nC[i] + G.nH[i], Nj = G.nC[j] + G.nH[j];
    return (min(G.cnt[i] + G.cnt[j], 15) << 2) | ((Ni == floor_(Ni) ? 1 : 0) << 1) | (Nj == floor_(Nj) ? 1 : 0);
}

// ------------------------------------------------------------------ REBO bonds
// EXTRA (here and in the torsion and b* kernels): the virial or the parameter
// gradient is wanted; the instances without them hold no accumulators for them.
template <class R, bool EXTRA>
__global__ void __launch_bounds__(128, 4) k_rebo(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, EXTRA && a.pgrad != nullptr, {0, 0, 0, 0, 0, 0}};
    // forward -> reverse angular terms (FP64: there they save FP64-pipe work;
    // the FP32 instances do better with the shared memory left to L1)
    __shared__ R scache[sizeof(R) == 8 ? side_cache_len<R>() * 128 : 1];
    SideCache<R> sc{sizeof(R) == 8 ? scache + threadIdx.x : nullptr, 128};
    double E = 0;
    // C-C, C-H, then H-H bonds (from the far end of a.bonds): warps of one species pair
    int ncc = min(*a.nccbonds, a.bond_cap), nch = min(*a.nbonds, a.bond_cap);
    int nhh = min(*a.nhhbonds, a.bond_cap - nch);
    int nb = ncc + nch + nhh;
    __shared__ int s_cnt[65], s_item[128];
    auto bond = [&](int b) {
        return b < ncc ? a.ccbonds[b] : (b < ncc + nch ? a.bonds[b - ncc] : a.bonds[a.bond_cap - 1 - (b - ncc - nch)]);
    };
    for (int base = blockIdx.x * 128; base < nb; base += gridDim.x * 128) {
        int b = base + threadIdx.x, key = -1;
        if (b < nb) {
            int2 bd = bond(b);
            key = bond_key<R>(a.G, bd.x, a.G.nj[bd.x * a.G.stride + bd.y]);
        }
        b = block_group<128>(key, b, s_cnt, s_item);
        if (b < 0) continue;
        int2 bd = bond(b);
        double e = rebo_bond<R>(P, a.G, bd.x, bd.y, sink, sc);
        E += e;
        if (a.eatom) eatom_pair(a.eatom, bd.x, a.G.nj[bd.x * a.G.stride + bd.y], e);
    }
    block_accumulate<128>(E, sink.W, EXTRA && a.virial, a.acc + 0, a.acc + 3);
}

// ------------------------------------------------------------------ torsion
template <class R, bool EXTRA>
__global__ void __launch_bounds__(128) k_torsion(StepArgs<R> a) {
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, EXTRA && a.pgrad != nullptr, {0, 0, 0, 0, 0, 0}};
    __shared__ R tstore[TORS_L * TORS_V * 128];        // the l-side values and sums of each thread
    TorsStore<R> S{tstore + threadIdx.x, 128};
    double E = 0;
    int nb = *a.nccbonds;
    if (nb > a.bond_cap) nb = a.bond_cap;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int2 bd = a.ccbonds[b];
        double e = torsion_bond_f<R>(P, a.G, bd.x, bd.y, sink, S);
        E += e;
        if (a.eatom && e != 0.0) eatom_pair(a.eatom, bd.x, a.G.nj[bd.x * a.G.stride + bd.y], e);
    }
    block_accumulate<128>(E, sink.W, EXTRA && a.virial, a.acc + 2, a.acc + 3);
}

// The torsion term in double-float on the FP64 short list (AIREBO_DF64): the
// term is short arithmetic on data the list already holds, which the FP32 pipe
// runs about three times faster than the FP64 pipe at FP64-class accuracy.
template <bool EXTRA>
__global__ void __launch_bounds__(128) k_torsion_dd(StepArgs<double> a) {
    const DevParams<dd>& P = *a.Pdd;
    GraphAs<dd, double> G(a.G);
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, false, {0, 0, 0, 0, 0, 0}};
    __shared__ dd tstore[TORS_L * TORS_V * 128];       // the l-side values and sums of each thread
    TorsStore<dd> S{tstore + threadIdx.x, 128};
    double E = 0;
    int nb = *a.nccbonds;
    if (nb > a.bond_cap) nb = a.bond_cap;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int2 bd = a.ccbonds[b];
        double e = torsion_bond_f<dd>(P, G, bd.x, bd.y, sink, S);
        E += e;
        if (a.eatom && e != 0.0) eatom_pair(a.eatom, bd.x, a.G.nj[bd.x * a.G.stride + bd.y], e);
    }
    block_accumulate<128>(E, sink.W, EXTRA && a.virial, a.acc + 2, a.acc + 3);
}

// ------------------------------------------------------------------ connectivity map
template <class R>
__global__ void __launch_bounds__(128) k_path_map(StepArgs<R> a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    PathMap<R> M = a.M;
    // the warp clears the hash tables of its atoms together: one contiguous
    // run of 16-byte stores
    {
        int i0 = i - (threadIdx.x & 31);
        int na = min(32, a.n - i0);
        if (na > 0) {
            uint4* T = reinterpret_cast<uint4*>(M.ht + ((size_t)i0 << M.hbits));
            int words = (na << M.hbits) / 2;
            for (int w = threadIdx.x & 31; w < words; w += 32) T[w] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncwarp();
    }
    if (i >= a.n) return;
    int ov = build_path_map<R>(a.G, M, i);
    if (ov) atomicMax(a.err + ERR_MAP, M.cnt[i] + ov);
}

// A slot in queue k (counter ctr[k]) for each lane of the warp that calls
// this: one atomic per distinct k among the calling lanes, which share it in
// lane order.  (An atomic on a per-lane address is not combined across the
// warp by the compiler, and 32 of them on one counter serialise.)
__device__ __forceinline__ int queue_slot(int* ctr, int k) {
    unsigned act = __activemask();
    unsigned peers = __match_any_sync(act, k);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(ctr + k, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1));
}

// ------------------------------------------------------------------ LJ
// Persistent warps stride over atoms i.  For each chunk of 32 entries of i's
// half list, every lane forms the FP64 displacement and tests its pair (cut-off,
// C_ij lookup, S_r); the pairs that need the full pair term are compacted with
// a ballot into a per-warp buffer in shared memory (the "compress" of Sec. 4.3),
// and the FP64 pair arithmetic runs only on full batches of 32 compacted pairs,
// so no lane idles through it.  Pairs with S_r != 0 go to the b* queue, pairs
// along a path (0 < C_ij < 1) to the queue of k_lj_path.
constexpr int LJ_THREADS = 256;
constexpr int LJ_WARPS = LJ_THREADS / 32;

// two compaction buffers per warp: 0 = inner pairs, 1 = pairs in the cut-off switch
struct LjBuf {
    int jp[2][64];          // j | species pair << 30
    int ia[2][64];          // the list's atom i
    int im[2][64];          // packed image of j
};

// Per-lane force (and energy) accumulator of the atom whose pairs the lane
// last evaluated.  Batches run across atom boundaries, so a lane flushes it
// with atomics when its next pair belongs to another atom.
struct LaneAcc {
    int own = -1;
    double fx = 0, fy = 0, fz = 0, e = 0;
    __device__ __forceinline__ void flush(double* f, int n, double* eatom) {
        if (own >= 0) {
            atomicAdd(f + own, fx); atomicAdd(f + n + own, fy); atomicAdd(f + 2 * n + own, fz);
            if (eatom) atomicAdd(eatom + own, e);
        }
        fx = fy = fz = e = 0;
    }
};

// FP64 displacement x_j + S L - x_i of a listed pair (minimum-image
// arithmetic stays double); shift holds S L for |S| <= 4 of a single box
template <class R>
__device__ __forceinline__ void lj_disp(const StepArgs<R>& a, const double (*shift)[9], int i, int j, int img,
                                        double& dx, double& dy, double& dz) {
    int n = a.n;
    dx = a.pos[j] - a.pos[i]; dy = a.pos[n + j] - a.pos[n + i]; dz = a.pos[2 * n + j] - a.pos[2 * n + i];
    if (img != 0) {
        int sx = img_x(img), sy = img_y(img), sz = img_z(img);
        if (a.sys || sx < -4 || sx > 4 || sy < -4 || sy > 4 || sz < -4 || sz > 4) {
            const double* L = box_of(a, i);
            dx += sx * L[0]; dy += sy * L[1]; dz += sz * L[2];
        } else {
            dx += shift[0][sx + 4]; dy += shift[1][sy + 4]; dz += shift[2][sz + 4];
        }
    }
}

template <class R>
__device__ __forceinline__ void lj_batch(const StepArgs<R>& a, const DevParams<R>& P, const double (*shift)[9],
                                         const LjPow* K, LjBuf& B, int b, int lane, Sink& sink, LaneAcc& acc,
                                         double& E) {
    int jp = B.jp[b][lane];
    int j = jp & 0x3fffffff, p = (unsigned)jp >> 30;
    int i = B.ia[b][lane];
    if (i != acc.own) {
        acc.flush(sink.f, sink.n, a.eatom);
        acc.own = i;
    }
    double dx, dy, dz;
    lj_disp<R>(a, shift, i, j, B.im[b][lane], dx, dy, dz);
    R rx = (R)dx, ry = (R)dy, rz = (R)dz;
    R r2 = rx * rx + ry * ry + rz * rz;
    double E0 = E;
    if (b == 0)
        lj_eval_inner<R>(K[p], j, dx, dy, dz, r2, sink, acc.fx, acc.fy, acc.fz, E);
    else
        lj_eval_switch<R>(P, K[p], p, j, dx, dy, dz, r2, sink, acc.fx, acc.fy, acc.fz, E);
    if (a.eatom) {
        acc.e += 0.5 * (E - E0);
        atomicAdd(a.eatom + j, 0.5 * (E - E0));
    }
}

// ---- double-float evaluation of the compacted pairs (precision AIREBO_DF64)
// Positions arrive split as hi + lo, hi rounded to a multiple of 2^-12 A (and
// |x| < 2000 A, so that hi has at most 23 significant bits): the difference
// of two such hi values, plus the same split of the image shift, is exact in
// FP32, so the displacement keeps FP64-class accuracy.  Pair forces go to
// 64-bit fixed-point sums (ff_to_fixed), added to the FP64 forces afterwards.
struct DfParams {
    ff sig2[3], eps4[3], swlo[3], swinv[3];
};

struct DfLaneAcc {
    int own = -1;
    long long fx = 0, fy = 0, fz = 0;            // fixed point, as the sums they go to
    ff e{0.0f, 0.0f};
    __device__ __forceinline__ void flush(unsigned long long* fix, int n, double* eatom) {
        if (own >= 0) {
            atomicAdd(fix + own, (unsigned long long)fx);
            atomicAdd(fix + n + own, (unsigned long long)fy);
            atomicAdd(fix + 2 * n + own, (unsigned long long)fz);
            if (eatom) atomicAdd(eatom + own, ff_to_double(e));
        }
        fx = fy = fz = 0;
        e = ff{0.0f, 0.0f};
    }
};

// Image shift S L of a split-position pair as hi + lo: from the table of the
// single box for |S| <= 4, from the system's split box edges for |S| <= 1
// (hi times -1, 0 or 1 stays exact), else split here in FP64 (tiny boxes)
template <class R>
__device__ __forceinline__ void shift_split(const StepArgs<R>& a, const float (*sh)[9], const float (*sl)[9],
                                            int i, int img, float* h, float* l) {
    int s3[3] = {img_x(img), img_y(img), img_z(img)};
    bool small = s3[0] >= -1 && s3[0] <= 1 && s3[1] >= -1 && s3[1] <= 1 && s3[2] >= -1 && s3[2] <= 1;
    if (!a.sys && s3[0] >= -4 && s3[0] <= 4 && s3[1] >= -4 && s3[1] <= 4 && s3[2] >= -4 && s3[2] <= 4) {
        for (int d = 0; d < 3; d++) { h[d] = sh[d][s3[d] + 4]; l[d] = sl[d][s3[d] + 4]; }
    } else if (small) {
        int sy = a.sys[i];
        float4 bh = a.Lhl[2 * sy], bl = a.Lhl[2 * sy + 1];
        h[0] = (float)s3[0] * bh.x; h[1] = (float)s3[1] * bh.y; h[2] = (float)s3[2] * bh.z;
        l[0] = (float)s3[0] * bl.x; l[1] = (float)s3[1] * bl.y; l[2] = (float)s3[2] * bl.z;
    } else {
        const double* L = box_of(a, i);
        for (int d = 0; d < 3; d++) df_split(s3[d] * L[d], h[d], l[d]);
    }
}

// the same as a called function: the double-float kernel is sensitive to its
// code size (instruction-cache stalls)
template <class R>
__device__ __noinline__ void shift_split_call(const StepArgs<R>& a, const float (*sh)[9], const float (*sl)[9],
                                              int i, int img, float* h, float* l) {
    shift_split<R>(a, sh, sl, i, img, h, l);
}

template <class R, bool EXTRA>
__device__ __noinline__ void lj_batch_df(const StepArgs<R>& a, const DfParams& D, const float (*sh)[9],
                                            const float (*sl)[9], LjBuf& B, int b, int lane, DfLaneAcc& acc,
                                            ff& E, ff* W) {
    int jp = B.jp[b][lane];
    int j = jp & 0x3fffffff, p = (unsigned)jp >> 30;
    int i = B.ia[b][lane];
    int img = B.im[b][lane];
    if (i != acc.own) {
        acc.flush(a.fix, a.n, a.eatom);
        acc.own = i;
    }
    float4 hi = a.posf[i], li = a.pq_lo[i], hj = a.posf[j], lj = a.pq_lo[j];
    float shx = 0.0f, shy = 0.0f, shz = 0.0f, slx = 0.0f, sly = 0.0f, slz = 0.0f;
    if (img != 0) {
        float h[3], l[3];
        shift_split_call<R>(a, sh, sl, i, img, h, l);
        shx = h[0]; shy = h[1]; shz = h[2]; slx = l[0]; sly = l[1]; slz = l[2];
    }
    // hi parts: exact (multiples of 2^-12 below 2^12 in magnitude); lo parts: rounded
    ff dx = two_sum(__fsub_rn(__fadd_rn(hj.x, shx), hi.x), __fsub_rn(__fadd_rn(lj.x, slx), li.x));
    ff dy = two_sum(__fsub_rn(__fadd_rn(hj.y, shy), hi.y), __fsub_rn(__fadd_rn(lj.y, sly), li.y));
    ff dz = two_sum(__fsub_rn(__fadd_rn(hj.z, shz), hi.z), __fsub_rn(__fadd_rn(lj.z, slz), li.z));
    ff r2 = ff_add(ff_add(ff_sqr(dx), ff_sqr(dy)), ff_sqr(dz));
    ff v, c;
    if (b == 0) {                 // C = 1, no path, r inside 2.7 sigma
        ff ir2 = ff_rcp(r2);
        ff s2 = ff_mul(D.sig2[p], ir2);
        ff s6 = ff_mul(ff_sqr(s2), s2);
        ff t = ff_mul(D.eps4[p], s6);                                   // 4 eps s6
        v = ff_mul(t, ff_add_f(s6, -1.0f));                             // 4 eps (s12 - s6)
        c = ff_mul(ff_mul(t, ff_add_f(ff_mul_f(s6, -12.0f), 6.0f)), ir2);   // (dV/dr) / r
    } else {                      // inside the cut-off switch
        ff ir = ff_rsqrt(r2);
        ff ir2 = ff_sqr(ir);
        ff s2 = ff_mul(D.sig2[p], ir2);
        ff s6 = ff_mul(ff_sqr(s2), s2);
        ff t = ff_mul(D.eps4[p], s6);
        ff vv = ff_mul(t, ff_add_f(s6, -1.0f));
        ff dvr = ff_mul(ff_mul(t, ff_add_f(ff_mul_f(s6, -12.0f), 6.0f)), ir2);
        ff r = ff_mul(r2, ir);
        ff x = ff_mul(ff_sub(r, D.swlo[p]), D.swinv[p]);                // > 0 in this class
        ff so = ff_add_f(ff_neg(ff_mul(ff_sqr(x), ff_add_f(ff_mul_f(x, -2.0f), 3.0f))), 1.0f);
        ff dso = ff_mul(ff_mul_f(ff_mul(x, ff_add_f(ff_neg(x), 1.0f)), -6.0f), D.swinv[p]);
        v = ff_mul(vv, so);
        c = ff_add(ff_mul(dvr, so), ff_mul(ff_mul(vv, dso), ir));
    }
    E = ff_add(E, v);
    if (a.eatom) {
        acc.e = ff_add(acc.e, ff_mul_f(v, 0.5f));
        atomicAdd(a.eatom + j, 0.5 * ff_to_double(v));
    }
    ff gx = ff_mul(c, dx), gy = ff_mul(c, dy), gz = ff_mul(c, dz);
    if (fabsf(gx.hi) < FIX_LIMIT && fabsf(gy.hi) < FIX_LIMIT && fabsf(gz.hi) < FIX_LIMIT) {
        long long qx = ff_to_fixed(gx), qy = ff_to_fixed(gy), qz = ff_to_fixed(gz);
        acc.fx += qx; acc.fy += qy; acc.fz += qz;
        atomicAdd(a.fix + j, (unsigned long long)(-qx));
        atomicAdd(a.fix + a.n + j, (unsigned long long)(-qy));
        atomicAdd(a.fix + 2 * a.n + j, (unsigned long long)(-qz));
    } else {
        atomicOr(a.err + ERR_DF, DF_FORCE);
    }
    if (EXTRA && a.virial) {
        W[0] = ff_sub(W[0], ff_mul(dx, gx)); W[1] = ff_sub(W[1], ff_mul(dy, gy)); W[2] = ff_sub(W[2], ff_mul(dz, gz));
        W[3] = ff_sub(W[3], ff_mul(dx, gy)); W[4] = ff_sub(W[4], ff_mul(dx, gz)); W[5] = ff_sub(W[5], ff_mul(dy, gz));
    }
}

// Mixed precision with the same split positions: the double-float
// displacement (FP64-class) rounded once to FP32, the pair term in FP32, and
// the pair forces summed in 64-bit fixed point, the energy and virial in
// double-float -- no FP64 instruction per pair.
template <class R, bool EXTRA>
__device__ __forceinline__ void lj_batch_mx(const StepArgs<R>& a, const DevParams<R>& P, const float (*sh)[9],
                                            const float (*sl)[9], LjBuf& B, int b, int lane, DfLaneAcc& acc,
                                            ff& E, ff* W) {
    int jp = B.jp[b][lane];
    int j = jp & 0x3fffffff, p = (unsigned)jp >> 30;
    int i = B.ia[b][lane];
    int img = B.im[b][lane];
    if (i != acc.own) {
        acc.flush(a.fix, a.n, a.eatom);
        acc.own = i;
    }
    float4 hi = a.posf[i], li = a.pq_lo[i], hj = a.posf[j], lj = a.pq_lo[j];
    float shx = 0.0f, shy = 0.0f, shz = 0.0f, slx = 0.0f, sly = 0.0f, slz = 0.0f;
    if (img != 0) {
        float h[3], l[3];
        shift_split<R>(a, sh, sl, i, img, h, l);
        shx = h[0]; shy = h[1]; shz = h[2]; slx = l[0]; sly = l[1]; slz = l[2];
    }
    float rx = __fadd_rn(__fsub_rn(__fadd_rn(hj.x, shx), hi.x), __fsub_rn(__fadd_rn(lj.x, slx), li.x));
    float ry = __fadd_rn(__fsub_rn(__fadd_rn(hj.y, shy), hi.y), __fsub_rn(__fadd_rn(lj.y, sly), li.y));
    float rz = __fadd_rn(__fsub_rn(__fadd_rn(hj.z, shz), hi.z), __fsub_rn(__fadd_rn(lj.z, slz), li.z));
    float r2 = rx * rx + ry * ry + rz * rz;
    float v, c;
    float sig2 = (float)P.sig2[p], e4 = (float)P.eps4[p];
    if (b == 0) {
        float ir2 = rcp_(r2);
        float s2 = sig2 * ir2;
        float s6 = s2 * s2 * s2;
        v = e4 * (s6 * s6 - s6);
        c = e4 * (6.0f * s6 - 12.0f * s6 * s6) * ir2;
    } else {
        float ir = rsqrt_(r2);
        float ir2 = ir * ir;
        float s2 = sig2 * ir2;
        float s6 = s2 * s2 * s2;
        float vv = e4 * (s6 * s6 - s6);
        float dvr = e4 * (-12.0f * s6 * s6 + 6.0f * s6) * ir2;
        float t = (r2 * ir - (float)P.swlo[p]) * (float)P.swinv[p];
        float so = 1.0f - t * t * (3.0f - 2.0f * t);
        float dso = -6.0f * t * (1.0f - t) * (float)P.swinv[p];
        v = vv * so;
        c = dvr * so + vv * dso * ir;
    }
    E = ff_add_f(E, v);
    if (a.eatom) {
        acc.e = ff_add_f(acc.e, 0.5f * v);
        atomicAdd(a.eatom + j, 0.5 * (double)v);
    }
    float gx = c * rx, gy = c * ry, gz = c * rz;
    if (fabsf(gx) < FIX_LIMIT && fabsf(gy) < FIX_LIMIT && fabsf(gz) < FIX_LIMIT) {
        long long qx = f2fix(gx), qy = f2fix(gy), qz = f2fix(gz);
        acc.fx += qx; acc.fy += qy; acc.fz += qz;
        atomicAdd(a.fix + j, (unsigned long long)(-qx));
        atomicAdd(a.fix + a.n + j, (unsigned long long)(-qy));
        atomicAdd(a.fix + 2 * a.n + j, (unsigned long long)(-qz));
    } else {
        atomicOr(a.err + ERR_DF, DF_FORCE);
    }
    if (EXTRA && a.virial) {
        W[0] = ff_add_f(W[0], -rx * gx); W[1] = ff_add_f(W[1], -ry * gy); W[2] = ff_add_f(W[2], -rz * gz);
        W[3] = ff_add_f(W[3], -rx * gy); W[4] = ff_add_f(W[4], -rx * gz); W[5] = ff_add_f(W[5], -ry * gz);
    }
}

// Pair tests on FP32 positions.  An FP32 squared distance r2f differs from
// the FP64 one by at most band (below); a test whose threshold lies within
// band of r2f is redone on the FP64 displacement, so every pair is classified
// exactly as the FP64 displacement classifies it.  Per component,
// |dx_f - dx| <= 2^-22 (2 max|x_i| + 4 |S|max L + 48): the roundings of x_i,
// x_j and S L to FP32 and of the two FP32 additions, with |x_j| <= |x_i| +
// |dx| + |S L| and |dx| < 16 A for any listed pair, and a factor 2 to spare.
//
// EXTRA: the virial or the parameter gradient is wanted.  The instance without
// them keeps no accumulators for them in registers (they cost the mixed
// instance its spill-free register budget).
template <class R, bool DF, int MODE>
__global__ void __launch_bounds__(LJ_THREADS, 4) k_lj(StepArgs<R> a) {
    constexpr bool EXTRA = MODE >= 1;      // virial or parameter gradient
    constexpr bool JV = MODE == 2;         // the parameter derivatives of the forces too
    const DevParams<R>& P = *a.P;
    __shared__ double shift[3][9];                // image shifts S L for S in [-4, 4]
    __shared__ LjCuts<float> cutsf[3];            // thresholds in FP32, by species pair
    __shared__ LjBuf bufs[LJ_WARPS];
    __shared__ float shf[2][3][9];                // DF: split image shifts (hi, lo)
    __shared__ DfParams dfp;
    __shared__ LjPow ljk[3];                       // the LJ pair in powers of 1/r^2, by species pair
    if (threadIdx.x < 27) {
        double v = (double)((int)(threadIdx.x % 9) - 4) * a.L[threadIdx.x / 9];
        shift[threadIdx.x / 9][threadIdx.x % 9] = v;
        if (DF) df_split(v, shf[0][threadIdx.x / 9][threadIdx.x % 9], shf[1][threadIdx.x / 9][threadIdx.x % 9]);
    }
    if (threadIdx.x < 3) {
        int q = threadIdx.x;
        cutsf[q] = LjCuts<float>{(float)P.rc2[q], (float)P.rpath2, (float)P.Srhi2[q], (float)P.swlo2[q]};
        ljk[q] = lj_pow((double)P.eps4[q], (double)P.sig2[q]);
        if (DF) {
            dfp.sig2[q] = ff_from_double((double)P.sig2[q]);
            dfp.eps4[q] = ff_from_double((double)P.eps4[q]);
            dfp.swlo[q] = ff_from_double((double)P.swlo[q]);
            dfp.swinv[q] = ff_from_double((double)P.swinv[q]);
        }
    }
    __syncthreads();
    int lane = threadIdx.x & 31;
    LjBuf& B = bufs[threadIdx.x >> 5];
    unsigned lt = (1u << lane) - 1u;
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, EXTRA && a.pgrad != nullptr, {0, 0, 0, 0, 0, 0}};
    bool general = EXTRA && (a.pgrad != nullptr || a.jv != nullptr);
    double J[6] = {0, 0, 0, 0, 0, 0};          // v . dF/d(eps, sigma) with a.jv
    LaneAcc acc;
    DfLaneAcc dacc;
    ff Edf{0.0f, 0.0f};
    ff Wdf[6] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    double E = 0;
    unsigned evaluated = 0;
    int n = a.n;
    int cnt[2] = {0, 0};
    // the pair arithmetic of one full (or, at the end, partial) batch
    auto batch = [&](int b) {
        if constexpr (DF) {
            if constexpr (sizeof(R) == 8) lj_batch_df<R, EXTRA>(a, dfp, shf[0], shf[1], B, b, lane, dacc, Edf, Wdf);
            else lj_batch_mx<R, EXTRA>(a, P, shf[0], shf[1], B, b, lane, dacc, Edf, Wdf);
        } else {
            lj_batch<R>(a, P, shift, ljk, B, b, lane, sink, acc, E);
        }
    };
    // warps take chunks of lj_chunk consecutive atoms from a global counter,
    // which balances C and H atoms (different list lengths) across warps; the
    // compaction buffers carry over from atom to atom, so that only the last
    // batch of a warp runs partly empty
    int chunk_end = 0;
    for (int i = 0;; i++) {
        if (i >= chunk_end) {
            int c = 0;
            if (lane == 0) c = atomicAdd(a.lj_next, a.lj_chunk);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= n) break;
            chunk_end = min(c + a.lj_chunk, n);
            i = c;
        }
        float4 pfi = a.posf[i];
        int ti = a.G.type[i];
        int ne = a.lj_cnt[i];
        const int2* row = a.lj + (size_t)i * a.lj_cap;
        const double* L = box_of(a, i);
        float Lf[3] = {(float)L[0], (float)L[1], (float)L[2]};
        float err0 = 2.0f * fmaxf(fabsf(pfi.x), fmaxf(fabsf(pfi.y), fabsf(pfi.z))) + 48.0f;
        float Lmax = fmaxf(Lf[0], fmaxf(Lf[1], Lf[2]));
        for (int base = 0; base < ne; base += 32) {
            int e = base + lane;
            int st = 0, j = 0, p = 0, img = 0;
            if (e < ne) {
                int2 ent = row[e];
                j = ent.x;
                img = ent.y;
                float4 pj = a.posf[j];
                float fx, fy, fz;
                float smax = 0.0f;
                if (DF) {             // hi parts on the 2^-12 grid: this difference is exact
                    float shx = 0.0f, shy = 0.0f, shz = 0.0f;
                    if (img != 0) {
                        float h[3], l[3];
                        if (sizeof(R) == 8) shift_split_call<R>(a, shf[0], shf[1], i, img, h, l);
                        else shift_split<R>(a, shf[0], shf[1], i, img, h, l);
                        shx = h[0]; shy = h[1]; shz = h[2];
                    }
                    fx = __fsub_rn(__fadd_rn(pj.x, shx), pfi.x);
                    fy = __fsub_rn(__fadd_rn(pj.y, shy), pfi.y);
                    fz = __fsub_rn(__fadd_rn(pj.z, shz), pfi.z);
                } else {
                    fx = pj.x - pfi.x; fy = pj.y - pfi.y; fz = pj.z - pfi.z;
                    if (img != 0) {
                        int sx = img_x(img), sy = img_y(img), sz = img_z(img);
                        fx += (float)sx * Lf[0]; fy += (float)sy * Lf[1]; fz += (float)sz * Lf[2];
                        smax = (float)max(abs(sx), max(abs(sy), abs(sz)));
                    }
                }
                float r2f = fx * fx + fy * fy + fz * fz;
                p = pidx(ti, __float_as_int(pj.w));
                LjCuts<float> kf = cutsf[p];
                // with split positions |dx - dx_hi| <= 3 * 2^-13 per component (the lo
                // parts and the shift's), so |r2f - r2| <= 3.7e-4 (2 sqrt(3) 16 + 1.1e-3)
                // plus the rounding of r2f
                float band;
                if (DF) {
                    band = 0.025f + 1e-6f * r2f;
                } else {
                    float err = 2.3841858e-7f * (err0 + 4.0f * smax * Lmax);      // 2^-22 (...)
                    band = err * (56.0f + 3.0f * err) + 1e-6f * r2f;
                }
                bool near = fabsf(r2f - kf.rc2) <= band || fabsf(r2f - kf.srhi2) <= band ||
                            fabsf(r2f - kf.swlo2) <= band || fabsf(r2f - kf.rpath2) <= band;
                R C;
                int code, mi;
                if (near) {                 // rare: decide on the FP64 displacement
                    double dx, dy, dz;
                    lj_disp<R>(a, shift, i, j, img, dx, dy, dz);
                    R rx = (R)dx, ry = (R)dy, rz = (R)dz;
                    R r2 = rx * rx + ry * ry + rz * rz;
                    evaluated += lt_nonneg(r2, P.rc2[p]);
                    st = lj_classify<R>(P, a.M, i, p, j, img, r2, C, code, mi, general);
                } else {
                    evaluated += r2f < kf.rc2;
                    st = lj_classify_c<R, float>(P, a.M, i, j, img, r2f, kf, C, code, mi, general);
                }
                if (st == 2) {
                    int q = queue_slot(a.nbq, p);
                    if (q < a.bq_cap) a.bq[(size_t)p * a.bq_cap + q] = make_int4(i, e, mi, 0);
                } else if (st == 4) {     // 0 < C < 1 along a path: to k_lj_path, a thread per pair
                    int q = queue_slot(a.npq, 0);
                    if (q < a.bq_cap) a.pq[q] = make_int4(i, e, mi, 0);
                }
            }
#pragma unroll
            for (int b = 0; b < 2; b++) {
                int want = b == 0 ? 1 : 3;
                unsigned m = __ballot_sync(0xffffffffu, st == want);
                if (st == want) {
                    int s = cnt[b] + __popc(m & lt);
                    B.jp[b][s] = j | (p << 30); B.ia[b][s] = i; B.im[b][s] = img;
                }
                cnt[b] += __popc(m);
                __syncwarp();
                if (cnt[b] >= 32) {
                    batch(b);
                    __syncwarp();
                    if (lane < cnt[b] - 32) {
                        int s = 32 + lane;
                        B.jp[b][lane] = B.jp[b][s]; B.ia[b][lane] = B.ia[b][s]; B.im[b][lane] = B.im[b][s];
                    }
                    cnt[b] -= 32;
                    __syncwarp();
                }
            }
        }
    }
    // the warp's last, partly filled batches
#pragma unroll
    for (int b = 0; b < 2; b++)
        if (lane < cnt[b]) batch(b);
    if (DF) {
        dacc.flush(a.fix, n, a.eatom);
        E += ff_to_double(Edf);
        if (EXTRA && a.virial)
            for (int k = 0; k < 6; k++) sink.W[k] += ff_to_double(Wdf[k]);
    } else {
        acc.flush(a.f, n, a.eatom);
    }
    unsigned ev = __reduce_add_sync(0xffffffffu, evaluated);
    if (lane == 0 && ev) atomicAdd(a.counters + CNT_LJ, (unsigned long long)ev);
    block_accumulate<LJ_THREADS>(E, sink.W, EXTRA && a.virial, a.acc + 1, a.acc + 3);
    if (EXTRA && a.pgrad) block_accumulate_g<LJ_THREADS>(sink.G, a.pgrad);
    if (JV && a.jv) block_accumulate_g<LJ_THREADS>(J, a.jout);
}

// The LJ pairs along a path (0 < C_ij < 1, or with the parameter derivatives
// every pair with C_ij > 0 outside the b* queue), queued by k_lj: a thread per
// pair, the general pair term with C_ij and the path's forces.  There are about one per atom once
// thermal motion makes partial bonds; evaluated inside k_lj, by the few lanes
// whose entries they were or in per-warp batches, they left most lanes of
// their FP64 instructions idle.
template <class R, int MODE>
__global__ void __launch_bounds__(128) k_lj_path(StepArgs<R> a) {
    constexpr bool EXTRA = MODE >= 1, JV = MODE == 2;
    const DevParams<R>& P = *a.P;
    __shared__ double shift[3][9];                // image shifts S L for S in [-4, 4]
    if (threadIdx.x < 27)
        shift[threadIdx.x / 9][threadIdx.x % 9] = (double)((int)(threadIdx.x % 9) - 4) * a.L[threadIdx.x / 9];
    __syncthreads();
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, EXTRA && a.pgrad != nullptr, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    double J[6] = {0, 0, 0, 0, 0, 0};          // v . dF/d(eps, sigma) with a.jv
    int n = a.n;
    int nq = min(*a.npq, a.bq_cap);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nq; u += gridDim.x * blockDim.x) {
        int4 q = a.pq[u];
        int i = q.x;
        int2 ent = a.lj[(size_t)i * a.lj_cap + q.y];
        int j = ent.x;
        int p = pidx(a.G.type[i], a.G.type[j]);
        R C = R(1);
        int code = -1;
        if (q.z >= 0) {
            C = a.M.wt[(size_t)i * a.M.cap + q.z];
            code = a.M.path[(size_t)i * a.M.cap + q.z];
        }
        double dx, dy, dz;
        lj_disp<R>(a, shift, i, j, ent.y, dx, dy, dz);
        double gx = 0, gy = 0, gz = 0, E0 = E;
        lj_eval<R>(P, a.G, i, p, j, dx, dy, dz, C, code, sink, gx, gy, gz, E);
        if (JV && a.jv) {                 // S_r = 0 here: E = C V
            R qx = (R)dx, qy = (R)dy, qz = (R)dz;
            lj_pair_jvp<R>(P, a.G, i, j, qx, qy, qz, qx * qx + qy * qy + qz * qz, C, code, R(0), R(0), a.jv, n, J);
        }
        atomicAdd(a.f + i, gx); atomicAdd(a.f + n + i, gy); atomicAdd(a.f + 2 * n + i, gz);
        if (a.eatom) eatom_pair(a.eatom, i, j, E - E0);
    }
    block_accumulate<128>(E, sink.W, EXTRA && a.virial, a.acc + 1, a.acc + 3);
    if (EXTRA && a.pgrad) block_accumulate_g<128>(sink.G, a.pgrad);
    if (JV && a.jv) block_accumulate_g<128>(J, a.jout);
}

// ------------------------------------------------------------------ b* pairs
// Phase 1: every queued pair.  b* enters the energy only through S_b, which is
// exactly 1 below b_min and 0 above b_max.  Where b* is clear of that
// transition, phase 1 finishes the pair; the others go to a second queue, and
// phase 2 evaluates them in one bond-order pass with its reverse.  In FP64 the
// phase-1 b* is an FP32 evaluation that carries a rigorous bound on its
// distance from the exact value, trusted only where that interval, widened by
// BSTAR_SCREEN_SLACK, lies clear of the transition (the screen).
template <class R>
__device__ __forceinline__ void bstar_load(const StepArgs<R>& a, int t, int& i, int& j, double& dx, double& dy,
                                           double& dz, R& C, int& code) {
    int4 q = a.bq[t];
    i = q.x;
    int2 ent = a.lj[(size_t)i * a.lj_cap + q.y];
    j = ent.x;
    load_disp(a.pos, a.n, box_of(a, i), i, j, ent.y, dx, dy, dz);
    C = R(1);
    code = -1;
    if (q.z >= 0) {
        C = a.M.wt[(size_t)i * a.M.cap + q.z];
        code = a.M.path[(size_t)i * a.M.cap + q.z];
    }
}

template <class R, int MODE>
// 64 registers (8 blocks of 128 per SM): this pass waits mostly on the
// gathers of the FP32 screen, and twice the warps of the compiler's own
// choice (80 registers) hide more of them (1.12 -> 1.03 ms at 1M PE, FP64)
__global__ void __launch_bounds__(128, 8) k_bstar(StepArgs<R> a) {
    constexpr bool EXTRA = MODE >= 1, JV = MODE == 2;
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, EXTRA && a.pgrad != nullptr, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    double J[6] = {0, 0, 0, 0, 0, 0};          // v . dF/d(eps, sigma) with a.jv
    // the screen's thresholds in FP32: b_min rounded down, b_max rounded up
    __shared__ float bcut[2][3];
    if (threadIdx.x < 3) {
        bcut[0][threadIdx.x] = __double2float_rd((double)P.bmin[threadIdx.x]);
        bcut[1][threadIdx.x] = __double2float_ru((double)P.bmax[threadIdx.x]);
    }
    __syncthreads();
    int n0 = min(a.nbq[0], a.bq_cap), n1 = min(a.nbq[1], a.bq_cap), n2 = min(a.nbq[2], a.bq_cap);
    int nq = n0 + n1 + n2;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nq; u += gridDim.x * blockDim.x) {
        // the queue is kept per species pair (CC, CH, HH), so that warps are uniform
        int t = u < n0 ? u : (u < n0 + n1 ? a.bq_cap + (u - n0) : 2 * a.bq_cap + (u - n0 - n1));
        int i, j, code;
        double dx, dy, dz;
        R C;
        bstar_load<R>(a, t, i, j, dx, dy, dz, C, code);
        R rx = (R)dx, ry = (R)dy, rz = (R)dz;
        R r2 = rx * rx + ry * ry + rz * rz;
        int p = pidx(a.G.type[i], a.G.type[j]);
        R Sb = R(0), dSb = R(1);
        bool decided = false, screened = false;
        if constexpr (sizeof(R) == 8) {
            if (a.screen) {
                // b* in FP32 with a bound e on its distance from the exact value:
                // S_b is exactly 1 or 0 when [b* - e, b* + e] lies below b_min or
                // above b_max (with room for the FP64 path's own rounding); the
                // interval's ends are rounded outwards, the thresholds inwards,
                // so the FP32 comparisons decide only what the exact ones would
                ef bs = bstar_value_ef(*a.Pef, GraphEf(a.G32), i, j, dx, dy, dz);
                float lo = __fsub_rd(__fsub_rd(bs.v, bs.e), BSTAR_SCREEN_SLACK);
                float hi = __fadd_ru(__fadd_ru(bs.v, bs.e), BSTAR_SCREEN_SLACK);
                bool below = hi < bcut[0][p];
                bool above = lo > bcut[1][p];
                decided = below || above;
                Sb = below ? R(1) : R(0);
                dSb = R(0);
                screened = true;
            }
        }
        if (!screened) {
            R bs = bstar_value<R>(P, a.G, i, j, rx, ry, rz, r2, sink);
            Sb = bstar_switch<R>(P, p, bs, dSb);
            decided = dSb == R(0);
        }
        if (decided) {
            double e = bstar_finish<R>(P, a.G, i, j, rx, ry, rz, r2, C, code, Sb, R(0), sink);
            E += e;
            if (a.eatom) eatom_pair(a.eatom, i, j, e);
            if (JV && a.jv) lj_pair_jvp<R>(P, a.G, i, j, rx, ry, rz, r2, C, code, Sb, R(0), a.jv, a.n, J);
        } else {
            int s = queue_slot(a.nbq2, p);            // kept by species pair, as the first queue
            if (s < a.bq_cap) a.bq2[(size_t)p * a.bq_cap + s] = t;
        }
    }
    block_accumulate<128>(E, sink.W, EXTRA && a.virial, a.acc + 1, a.acc + 3);
    if (EXTRA && a.pgrad) block_accumulate_g<128>(sink.G, a.pgrad);
    if (JV && a.jv) block_accumulate_g<128>(J, a.jout);
}

// Phase 2: the pairs of the second queue, b* and its gradient in one pass.
// The FP32 (mixed) instance at 5 blocks per SM (0.655 -> 0.613 ms at 1M PE);
// the FP64 one is best at 4 (3.0 ms; 3 and 5 blocks: 3.6 and 3.1 ms).
template <class R, int MODE>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 5 : 4) k_bstar_rev(StepArgs<R> a) {
    constexpr bool EXTRA = MODE >= 1, JV = MODE == 2;
    const DevParams<R>& P = *a.P;
    Sink sink{a.f, a.n, EXTRA && a.virial, {0, 0, 0, 0, 0, 0}, EXTRA && a.pgrad != nullptr, {0, 0, 0, 0, 0, 0}};
    double E = 0;
    double J[6] = {0, 0, 0, 0, 0, 0};          // v . dF/d(eps, sigma) with a.jv
    unsigned dsb_count = 0;
    // forward -> reverse angular terms (FP64: there they save FP64-pipe work;
    // the FP32 instances do better with the shared memory left to L1)
    __shared__ R scache[sizeof(R) == 8 ? side_cache_len<R>() * 128 : 1];
    SideCache<R> sc{sizeof(R) == 8 ? scache + threadIdx.x : nullptr, 128};
    int n0 = min(a.nbq2[0], a.bq_cap), n1 = min(a.nbq2[1], a.bq_cap), n2 = min(a.nbq2[2], a.bq_cap);
    int nq = n0 + n1 + n2;
    // species pair by species pair (CC, CH, HH); in FP64 each block's pairs are
    // further grouped by the two atoms' neighbour counts and whether their
    // coordinations are integers (the spline knot paths), so that the lanes of
    // a warp run like bond orders (the FP32 instance is faster without)
    __shared__ int s_cnt[65], s_item[128];
    auto seg = [&](int u) { return u < n0 ? u : (u < n0 + n1 ? a.bq_cap + (u - n0) : 2 * a.bq_cap + (u - n0 - n1)); };
    constexpr bool GROUP = sizeof(R) == 8;
    int step = GROUP ? gridDim.x * 128 : gridDim.x * blockDim.x;
    for (int base = blockIdx.x * (GROUP ? 128 : blockDim.x); base < nq; base += step) {
        int u = base + (GROUP ? threadIdx.x : 0);
        if constexpr (GROUP) {
            int key = -1;
            if (u < nq) {
                int4 q = a.bq[a.bq2[seg(u)]];
                key = bond_key<R>(a.G, q.x, a.lj[(size_t)q.x * a.lj_cap + q.y].x);
            }
            u = block_group<128>(key, u, s_cnt, s_item);
            if (u < 0) continue;
        } else {
            u = base + threadIdx.x;
            if (u >= nq) break;
        }
        int s = seg(u);
        int i, j, code;
        double dx, dy, dz;
        R C;
        bstar_load<R>(a, a.bq2[s], i, j, dx, dy, dz, C, code);
        R rx = (R)dx, ry = (R)dy, rz = (R)dz;
        R r2 = rx * rx + ry * ry + rz * rz;
        bool dsb;
        double e = bstar_full<R>(P, a.G, i, j, rx, ry, rz, r2, C, code, sink, dsb, sc);
        dsb_count += dsb;
        E += e;
        if (a.eatom) eatom_pair(a.eatom, i, j, e);
        if (JV && a.jv) {
            R Sb;
            R dotSb = bstar_jvp<R>(P, a.G, i, j, rx, ry, rz, r2, a.jv, a.n, Sb);
            lj_pair_jvp<R>(P, a.G, i, j, rx, ry, rz, r2, C, code, Sb, dotSb, a.jv, a.n, J);
        }
    }
    unsigned c = __reduce_add_sync(0xffffffffu, dsb_count);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(a.counters + CNT_DSB, (unsigned long long)c);
    block_accumulate<128>(E, sink.W, EXTRA && a.virial, a.acc + 1, a.acc + 3);
    if (EXTRA && a.pgrad) block_accumulate_g<128>(sink.G, a.pgrad);
    if (JV && a.jv) block_accumulate_g<128>(J, a.jout);
}

template <class R>
__global__ void k_finish_counters(StepArgs<R> a) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        a.counters[CNT_BONDS] = (unsigned long long)(*a.nbonds + *a.nccbonds + *a.nhhbonds);
        a.counters[CNT_BSTAR] = (unsigned long long)(a.nbq[0] + a.nbq[1] + a.nbq[2]);
        a.counters[CNT_BSTAR_FULL] = (unsigned long long)(a.nbq2[0] + a.nbq2[1] + a.nbq2[2]);
        // the longest b* queue, kept with the other flags (a capacity check
        // after several asynchronous evaluations sees the largest of them)
        int q = max(max(a.nbq[0], a.nbq[1]), max(a.nbq[2], *a.npq));
        if (q > a.bq_cap) atomicMax(a.err + ERR_QUEUE, q);
    }
}

// Check of the screen's bound on every queued b* pair: the FP64 b* against
// the bounded FP32 one.  out (double[6], zeroed): pairs with a finite bound,
// pairs with an infinite one, the largest |b*_32 - b*_64| / bound, the
// largest bound, pairs where the difference exceeds the bound, and the
// largest difference.
static __global__ void __launch_bounds__(128) k_bstar_bound_check(StepArgs<double> a, double* out) {
    const DevParams<double>& P = *a.P;
    Sink none{nullptr, 0, false, {0, 0, 0, 0, 0, 0}, false, {0, 0, 0, 0, 0, 0}};
    int n0 = min(a.nbq[0], a.bq_cap), n1 = min(a.nbq[1], a.bq_cap), n2 = min(a.nbq[2], a.bq_cap);
    int nq = n0 + n1 + n2;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nq; u += gridDim.x * blockDim.x) {
        int t = u < n0 ? u : (u < n0 + n1 ? a.bq_cap + (u - n0) : 2 * a.bq_cap + (u - n0 - n1));
        int i, j, code;
        double dx, dy, dz, C;
        bstar_load<double>(a, t, i, j, dx, dy, dz, C, code);
        double b64 = bstar_value<double>(P, a.G, i, j, dx, dy, dz, dx * dx + dy * dy + dz * dz, none);
        ef bs = bstar_value_ef(*a.Pef, GraphEf(a.G32), i, j, dx, dy, dz);
        double diff = fabs((double)bs.v - b64);
        if (!(bs.e < EF_INF)) { atomicAdd(out + 1, 1.0); continue; }
        atomicAdd(out + 0, 1.0);
        double e = (double)bs.e;
        atomicMax((unsigned long long*)(out + 2), (unsigned long long)__double_as_longlong(e > 0 ? diff / e : (diff > 0 ? 1e300 : 0.0)));
        atomicMax((unsigned long long*)(out + 3), (unsigned long long)__double_as_longlong(e));
        if (diff > e) atomicAdd(out + 4, 1.0);
        atomicMax((unsigned long long*)(out + 5), (unsigned long long)__double_as_longlong(diff));
    }
}

// the fixed-point LJ force sums of the double-float kernel into the FP64
// forces (the sums are cleared before each evaluation)
static __global__ void k_fix_add(unsigned long long* fix, double* f, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < 3; d++) f[d * n + i] += (double)(long long)fix[d * n + i] * FIX_INV;
}

template <class R>
void launch_compute_impl(const StepArgs<R>& a, cudaStream_t s, int num_sms, cudaEvent_t* ev) {
    if (a.n == 0) return;
    int n = a.n;
    auto mark = [&](int k) { if (ev) cudaEventRecord(ev[k], s); };
    // grid-stride kernels launch whole waves: waves x resident blocks per SM x SMs
    // (the occupancies are asked once; nothing but stream work during graph capture)
    // mode 0: plain evaluation; 1: with the virial or the parameter gradient;
    // 2: with the parameter derivatives of the forces (LJ and b* kernels)
    int mode = a.jv ? 2 : ((a.virial || a.pgrad != nullptr) ? 1 : 0);
    bool extra = mode >= 1;
    static int occ_all[3][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}};
    int* occ = occ_all[mode];
    if (occ[0] < 0) {
        if (extra) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_rebo<R, true>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_torsion<R, true>, 128, 0);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_rebo<R, false>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_torsion<R, false>, 128, 0);
        }
        if (mode == 2) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_bstar<R, 2>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[3], k_bstar_rev<R, 2>, 128, 0);
        } else if (mode == 1) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_bstar<R, 1>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[3], k_bstar_rev<R, 1>, 128, 0);
        } else {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], k_bstar<R, 0>, 128, 0);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[3], k_bstar_rev<R, 0>, 128, 0);
        }
    }
    auto grid_of = [&](int k, int waves) { return num_sms * (occ[k] > 0 ? occ[k] : 1) * waves; };
    mark(0);
    k_posf<R><<<(n + 127) / 128, 128, 0, s>>>(a);
    k_short_list<R><<<(n + 127) / 128, 128, 0, s>>>(a);
    mark(1);
    if (a.rebo) {
        if (extra) k_rebo<R, true><<<grid_of(0, a.bond_waves), 128, 0, s>>>(a);
        else k_rebo<R, false><<<grid_of(0, a.bond_waves), 128, 0, s>>>(a);
    }
    mark(2);
    if (a.torsion) {
        bool dd_torsion = false;
        if constexpr (std::is_same<R, double>::value) {
            if (a.Pdd) {
                static int occ_dd[2] = {-1, -1};
                int& o = occ_dd[extra];
                if (o < 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, extra ? k_torsion_dd<true> : k_torsion_dd<false>, 128, 0);
                int g = num_sms * (o > 0 ? o : 1) * a.bond_waves;
                if (extra) k_torsion_dd<true><<<g, 128, 0, s>>>(a);
                else k_torsion_dd<false><<<g, 128, 0, s>>>(a);
                dd_torsion = true;
            }
        }
        if (!dd_torsion) {
            if (extra) k_torsion<R, true><<<grid_of(1, a.bond_waves), 128, 0, s>>>(a);
            else k_torsion<R, false><<<grid_of(1, a.bond_waves), 128, 0, s>>>(a);
        }
    }
    mark(3);
    if (a.lj_on) k_path_map<R><<<(n + 127) / 128, 128, 0, s>>>(a);
    mark(4);
    if (a.lj_on) {
        // asked once: nothing but stream work during graph capture
        static int per_sm[6] = {-1, -1, -1, -1, -1, -1};
        bool df = a.fix != nullptr;
        int need = (n + LJ_WARPS - 1) / LJ_WARPS;
        auto launch = [&](auto kernel, int slot) {
            if (per_sm[slot] < 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[slot], kernel, LJ_THREADS, 0);
            int blocks = num_sms * (per_sm[slot] > 0 ? per_sm[slot] : 1);
            kernel<<<blocks < need ? blocks : need, LJ_THREADS, 0, s>>>(a);
        };
        if (df) {
            if (mode == 2) launch(k_lj<R, true, 2>, 5);
            else if (mode == 1) launch(k_lj<R, true, 1>, 3);
            else launch(k_lj<R, true, 0>, 2);
            k_fix_add<<<(n + 255) / 256, 256, 0, s>>>(a.fix, a.f, n);
        } else {
            if (mode == 2) launch(k_lj<R, false, 2>, 4);
            else if (mode == 1) launch(k_lj<R, false, 1>, 1);
            else launch(k_lj<R, false, 0>, 0);
        }
        {                                 // the pairs along a path that k_lj queued
            int g = num_sms * 16;
            if (mode == 2) k_lj_path<R, 2><<<g, 128, 0, s>>>(a);
            else if (mode == 1) k_lj_path<R, 1><<<g, 128, 0, s>>>(a);
            else k_lj_path<R, 0><<<g, 128, 0, s>>>(a);
        }
    }
    mark(5);
    if (a.lj_on) {
        int g = grid_of(2, a.bstar_waves);
        if (mode == 2) k_bstar<R, 2><<<g, 128, 0, s>>>(a);
        else if (mode == 1) k_bstar<R, 1><<<g, 128, 0, s>>>(a);
        else k_bstar<R, 0><<<g, 128, 0, s>>>(a);
    }
    mark(6);
    if (a.lj_on) {
        int g = grid_of(3, a.bstar_waves);
        if (mode == 2) k_bstar_rev<R, 2><<<g, 128, 0, s>>>(a);
        else if (mode == 1) k_bstar_rev<R, 1><<<g, 128, 0, s>>>(a);
        else k_bstar_rev<R, 0><<<g, 128, 0, s>>>(a);
    }
    mark(7);
    k_finish_counters<R><<<1, 32, 0, s>>>(a);
}

}  // namespace airebo
