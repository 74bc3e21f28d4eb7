// Neighbour lists by binning (Sec. 2) and the velocity-Verlet step.
//
// Atoms are binned into cells at least half a long cut-off wide and counting-
// sorted by cell.  One thread per sorted atom then scans the cells of the
// stencil, with explicit periodic images (boxes may be smaller than twice the
// cut-off), and writes
//   - a half list of pairs with r < 3 sigma_ij + skin for the LJ term, and
//   - a full intermediate list with r < Dmax_ij + skin, from which the exact
//     REBO list is filtered every step (Sec. 4.1).
// The distance test runs in FP32 on wrapped coordinates with a small safety
// margin: the lists are supersets, every compute kernel applies the exact
// cut-off in FP64.  Each entry stores the neighbour and its image S relative
// to the caller's (unwrapped) positions: x_j + S L - x_i.
#include "internal.h"

namespace airebo {

// the cell grid an atom is binned on: the single system's, or its system's
struct Grid {
    int nc[3], reach[3], cell0;
    double cw[3], L[3];
};
__device__ __forceinline__ Grid grid_of(const NeighborArgs& a, int i) {
    Grid g;
    if (!a.sys) {
        for (int d = 0; d < 3; d++) { g.nc[d] = a.nc[d]; g.reach[d] = a.reach[d]; g.cw[d] = a.cell_w[d]; g.L[d] = a.L[d]; }
        g.cell0 = 0;
    } else {
        int s = a.sys[i];
        for (int d = 0; d < 3; d++) {
            g.nc[d] = a.snc[3 * s + d]; g.reach[d] = a.sreach[3 * s + d];
            g.cw[d] = a.scw[3 * s + d]; g.L[d] = a.Lsys[3 * s + d];
        }
        g.cell0 = a.scell0[s];
    }
    return g;
}

// a gated build (a.gate set) runs only when the device decided to rebuild
__device__ __forceinline__ bool gated_off(const int* gate) { return gate && *gate == 0; }

__global__ void k_bin(NeighborArgs a) {
    if (gated_off(a.gate)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    Grid g = grid_of(a, i);
    int c[3];
    for (int d = 0; d < 3; d++) {
        double x = a.pos[d * a.n + i];
        if (!isfinite(x)) { atomicMax(a.err + 2, 1); x = 0.0; }
        double w = floor(x / g.L[d]);
        if (w < -120.0 || w > 120.0) { atomicMax(a.err + 2, 2); w = 0.0; }
        double xw = x - w * g.L[d];
        int cd = (int)(xw / g.cw[d]);
        c[d] = cd < 0 ? 0 : (cd >= g.nc[d] ? g.nc[d] - 1 : cd);
    }
    int cell = g.cell0 + (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
    if (a.type[i] != 0 && a.type[i] != 1) atomicMax(a.err + 3, 1);
    a.cell_of[i] = cell;
    atomicAdd(a.cell_count + cell, 1);
}

// exclusive scan of the cell counts, one block
// Exclusive scan of the cell counts into the cell starts (and the fill
// cursors), by one block over tiles of 1024 cells: coalesced loads, a
// shuffle scan in each warp, then over the warps' sums, and a running carry.
__global__ void __launch_bounds__(1024) k_scan(const int* count, int* start, int* fill, int ncell, const int* gate) {
    if (gated_off(gate)) return;
    __shared__ int wsum[32];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int carry = 0;
    for (int base = 0; base < ncell; base += 1024) {
        int c = base + t;
        int v = c < ncell ? count[c] : 0;
        int x = v;                                   // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {                                // inclusive scan of the 32 warp sums
            int y = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            wsum[lane] = y;
        }
        __syncthreads();
        int excl = carry + (w > 0 ? wsum[w - 1] : 0) + x - v;
        if (c < ncell) {
            start[c] = excl;
            fill[c] = excl;
        }
        carry += wsum[31];
        __syncthreads();                             // wsum is rewritten by the next tile
    }
    if (t == 0) start[ncell] = carry;
}

__global__ void k_scatter(NeighborArgs a) {
    if (gated_off(a.gate)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int slot = atomicAdd(a.cell_fill + a.cell_of[i], 1);
    Grid g = grid_of(a, i);
    float xw[3];
    int wr[3];
    for (int d = 0; d < 3; d++) {
        double x = a.pos[d * a.n + i];
        if (!isfinite(x)) x = 0.0;
        double w = floor(x / g.L[d]);
        if (w < -120.0 || w > 120.0) w = 0.0;
        xw[d] = (float)(x - w * g.L[d]);
        wr[d] = (int)w;
    }
    // the fourth word: the atom and its species (bit 30), so that the list
    // build reads one float4 per tested candidate
    a.spos[slot] = make_float4(xw[0], xw[1], xw[2], __int_as_float(i | ((a.type[i] == 1 ? 1 : 0) << 30)));
    a.swrap[slot] = make_char4((char)wr[0], (char)wr[1], (char)wr[2], (char)(a.type[i] == 1 ? 1 : 0));
}

__global__ void __launch_bounds__(128) k_build(NeighborArgs a, const int* cell_start) {
    if (gated_off(a.gate)) return;
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n) return;
    float4 pi = a.spos[s];
    char4 wi = a.swrap[s];
    int i = __float_as_int(pi.w) & 0x3fffffff;
    int ti = wi.w;
    Grid g = grid_of(a, i);
    int cell = a.cell_of[i] - g.cell0;
    int ci[3] = {cell / (g.nc[1] * g.nc[2]), (cell / g.nc[2]) % g.nc[1], cell % g.nc[2]};
    float lj2[2], im2[2];
    for (int t = 0; t < 2; t++) {
        lj2[t] = a.lj_rc[ti + t] * a.lj_rc[ti + t];
        im2[t] = a.im_rc[ti + t] * a.im_rc[ti + t];
    }
    // cells farther than the largest cut-off from this atom are skipped: the
    // squared distance from the atom to a stencil cell's box, per dimension
    float rmax2 = fmaxf(fmaxf(lj2[0], lj2[1]), fmaxf(im2[0], im2[1]));
    float rim2 = fmaxf(im2[0], im2[1]);
    float Lf[3] = {(float)g.L[0], (float)g.L[1], (float)g.L[2]};
    float cwf[3] = {(float)g.cw[0], (float)g.cw[1], (float)g.cw[2]};
    int nlj = 0, nim = 0;
    int2* ljrow = a.lj + (size_t)i * a.lj_cap;
    int2* imrow = a.im + (size_t)i * a.im_cap;
    // distance from the atom to the slab [q w, (q + 1) w) of stencil cell q (margin 2e-3 A)
    auto slab = [&](int q, int d, float p) {
        float lo = q * cwf[d] - p, hi = lo + cwf[d];
        float e = lo > 0.0f ? lo : (hi < 0.0f ? -hi : 0.0f);
        e = fmaxf(e - 2e-3f, 0.0f);
        return e * e;
    };
    for (int ox = -g.reach[0]; ox <= g.reach[0]; ox++) {
        int qx = ci[0] + ox;
        float ex = slab(qx, 0, pi.x);
        if (ex >= rmax2) continue;
        int sx = qx >= 0 ? qx / g.nc[0] : -((-qx + g.nc[0] - 1) / g.nc[0]);
        int cx = qx - sx * g.nc[0];
        for (int oy = -g.reach[1]; oy <= g.reach[1]; oy++) {
            int qy = ci[1] + oy;
            float ey = ex + slab(qy, 1, pi.y);
            if (ey >= rmax2) continue;
            int sy = qy >= 0 ? qy / g.nc[1] : -((-qy + g.nc[1] - 1) / g.nc[1]);
            int cy = qy - sy * g.nc[1];
            for (int oz = -g.reach[2]; oz <= g.reach[2]; oz++) {
                int qz = ci[2] + oz;
                float ez = ey + slab(qz, 2, pi.z);
                if (ez >= rmax2) continue;
                int sz = qz >= 0 ? qz / g.nc[2] : -((-qz + g.nc[2] - 1) / g.nc[2]);
                int cz = qz - sz * g.nc[2];
                int c = g.cell0 + (cx * g.nc[1] + cy) * g.nc[2] + cz;
                float shx = sx * Lf[0] - pi.x, shy = sy * Lf[1] - pi.y, shz = sz * Lf[2] - pi.z;
                // the LJ half list keeps a pair in the row of the atom that
                // sorts first (cell order): beyond the REBO range only the
                // candidates sorted from this atom on can enter a list
                int e1 = cell_start[c + 1];
                int t0 = ez < rim2 ? cell_start[c] : max(cell_start[c], s);
                for (int t = t0; t < e1; t++) {
                    float4 pj = a.spos[t];
                    float dx = pj.x + shx, dy = pj.y + shy, dz = pj.z + shz;
                    float r2 = dx * dx + dy * dy + dz * dz;
                    int jt = __float_as_int(pj.w);
                    int tj = jt >> 30;
                    if (r2 >= lj2[tj]) continue;
                    int j = jt & 0x3fffffff;
                    char4 wj = a.swrap[t];
                    int Sx = sx - wj.x + wi.x, Sy = sy - wj.y + wi.y, Sz = sz - wj.z + wi.z;
                    bool self = (j == i);
                    if (self && Sx == 0 && Sy == 0 && Sz == 0) continue;
                    int img = pack_img(Sx, Sy, Sz);
                    if (r2 < im2[tj]) {
                        if (nim < a.im_cap) imrow[nim] = make_int2(j, img);
                        nim++;
                    }
                    bool pos = Sx > 0 || (Sx == 0 && (Sy > 0 || (Sy == 0 && Sz > 0)));
                    if (a.with_lj && (t > s || (self && pos))) {
                        if (nlj < a.lj_cap) ljrow[nlj] = make_int2(j, img);
                        nlj++;
                    }
                }
            }
        }
    }
    a.lj_cnt[i] = nlj < a.lj_cap ? nlj : a.lj_cap;
    a.im_cnt[i] = nim < a.im_cap ? nim : a.im_cap;
    if (nlj > a.lj_cap) atomicMax(a.err + 0, nlj);
    if (nim > a.im_cap) atomicMax(a.err + 1, nim);
}

// Carbon neighbours first in each intermediate REBO row, so that the exact
// REBO slots of every atom come out carbon-first too: the threads of a bond
// kernel then meet the species of the neighbours k in the same slot order
// and run the same branches.  (Two-pointer partition; rows are short.)
__global__ void k_order_im(NeighborArgs a) {
    if (gated_off(a.gate)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int c = min(a.im_cnt[i], a.im_cap);
    int2* row = a.im + (size_t)i * a.im_cap;
    int lo = 0, hi = c - 1;
    while (lo < hi) {
        while (lo < hi && a.type[row[lo].x] == 0) lo++;
        while (lo < hi && a.type[row[hi].x] != 0) hi--;
        if (lo < hi) {
            int2 t = row[lo];
            row[lo] = row[hi];
            row[hi] = t;
            lo++;
            hi--;
        }
    }
}

void launch_neighbor(NeighborArgs& a, cudaStream_t s, int ncell) {
    if (a.n == 0) return;
    cudaMemsetAsync(a.cell_count, 0, sizeof(int) * ncell, s);
    int nb = (a.n + 127) / 128;
    k_bin<<<nb, 128, 0, s>>>(a);
    k_scan<<<1, 1024, 0, s>>>(a.cell_count, a.cell_start, a.cell_fill, ncell, a.gate);
    k_scatter<<<nb, 128, 0, s>>>(a);
    k_build<<<nb, 128, 0, s>>>(a, a.cell_start);
    k_order_im<<<nb, 128, 0, s>>>(a);
}

__global__ void k_clear_cells(int* count, int ncell, const int* gate) {
    if (gated_off(gate)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) count[c] = 0;
}

// the positions of the build, for the next displacement check
__global__ void k_copy_ref(const double* pos, double* xref, int n3, const int* gate) {
    if (gated_off(gate)) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += gridDim.x * blockDim.x) xref[k] = pos[k];
}

void launch_neighbor_gated(NeighborArgs& a, cudaStream_t s, int ncell) {
    if (a.n == 0) return;
    int nb = (a.n + 127) / 128;
    k_clear_cells<<<(ncell + 255) / 256, 256, 0, s>>>(a.cell_count, ncell, a.gate);
    k_bin<<<nb, 128, 0, s>>>(a);
    k_scan<<<1, 1024, 0, s>>>(a.cell_count, a.cell_start, a.cell_fill, ncell, a.gate);
    k_scatter<<<nb, 128, 0, s>>>(a);
    k_build<<<nb, 128, 0, s>>>(a, a.cell_start);
    k_order_im<<<nb, 128, 0, s>>>(a);
    k_copy_ref<<<(3 * a.n + 255) / 256, 256, 0, s>>>(a.pos, a.xref, 3 * a.n, a.gate);
}

__global__ void k_rebuild_decide(const unsigned long long* maxd2, double half2, int* gate, long long* builds) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int g = __longlong_as_double((long long)*maxd2) > half2 ? 1 : 0;
        *gate = g;
        if (g) *builds += 1;
    }
}

void launch_rebuild_decide(const unsigned long long* maxd2, double half2, int* gate, long long* builds, cudaStream_t s) {
    k_rebuild_decide<<<1, 32, 0, s>>>(maxd2, half2, gate, builds);
}

// per-system energy: sum of the per-atom energies of each system's atoms
__global__ void k_system_energy(const double* eatom, const long long* off, double* out) {
    __shared__ double red[8];
    int s = blockIdx.x;
    double e = 0;
    for (long long i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) e += eatom[i];
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[s] = t;
    }
}

void launch_system_energy(const double* eatom, const long long* offsets, int nsys, double* out, cudaStream_t s) {
    if (nsys > 0) k_system_energy<<<nsys, 256, 0, s>>>(eatom, offsets, out);
}

// ------------------------------------------------------------------ NVE
constexpr double MVV2E = 103.642697;          // amu A^2 / fs^2 in eV

__global__ void k_nve_half(double* pos, double* vel, const double* f, const int8_t* type, int n, double dt,
                           bool drift, const double* xref, unsigned long long* maxd2, double* ke) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double k = 0, d2 = 0;
    if (i < n) {
        double m = type[i] == 0 ? 12.011 : 1.008;
        double c = 0.5 * dt / (m * MVV2E);
        double vx = vel[i] + c * f[i];
        double vy = vel[n + i] + c * f[n + i];
        double vz = vel[2 * n + i] + c * f[2 * n + i];
        vel[i] = vx; vel[n + i] = vy; vel[2 * n + i] = vz;
        if (drift) {
            double x = pos[i] + dt * vx, y = pos[n + i] + dt * vy, z = pos[2 * n + i] + dt * vz;
            pos[i] = x; pos[n + i] = y; pos[2 * n + i] = z;
            double ex = x - xref[i], ey = y - xref[n + i], ez = z - xref[2 * n + i];
            d2 = ex * ex + ey * ey + ez * ez;
            if (!(d2 == d2)) d2 = 1e300;
        }
        k = 0.5 * m * MVV2E * (vx * vx + vy * vy + vz * vz);
    }
    if (drift && maxd2) {
        for (int o = 16; o > 0; o >>= 1) d2 = fmax(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        if ((threadIdx.x & 31) == 0) atomicMax(maxd2, (unsigned long long)__double_as_longlong(d2));
    }
    if (ke) {
        for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(ke, k);
    }
}

__global__ void k_max_disp(const double* pos, const double* xref, int n, unsigned long long* maxd2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0;
    if (i < n) {
        double ex = pos[i] - xref[i], ey = pos[n + i] - xref[n + i], ez = pos[2 * n + i] - xref[2 * n + i];
        d2 = ex * ex + ey * ey + ez * ez;
        if (!(d2 == d2)) d2 = 1e300;
    }
    for (int o = 16; o > 0; o >>= 1) d2 = fmax(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxd2, (unsigned long long)__double_as_longlong(d2));
}

void launch_nve_half(double* pos, double* vel, const double* f, const int8_t* type, int n, double dt, bool drift,
                     const double* xref, unsigned long long* maxd2, double* ke, cudaStream_t s) {
    if (n == 0) return;
    k_nve_half<<<(n + 255) / 256, 256, 0, s>>>(pos, vel, f, type, n, dt, drift, xref, maxd2, ke);
}

void launch_max_disp(const double* pos, const double* xref, int n, unsigned long long* maxd2, cudaStream_t s) {
    if (n == 0) return;
    k_max_disp<<<(n + 255) / 256, 256, 0, s>>>(pos, xref, n, maxd2);
}

}  // namespace airebo
