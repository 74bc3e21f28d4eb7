// Declarations shared by the translation units of libairebo (not public).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include "terms.cuh"

namespace airebo {

// per-step device data of one precision R, all owned by the handle
template <class R> struct StepBuffers {
    DevParams<R>* P = nullptr;        // device copy of the parameter struct
    DevParams<R>* Pkg = nullptr;      // the same with the spline-gradient buffer set (knot gradients)
    R* tables = nullptr;              // P, pi^rc and T coefficients
    unsigned char* Tnz = nullptr;
    // short list
    int* cnt = nullptr; int* nj = nullptr; int* nimg = nullptr;
    R* dx = nullptr; R* dy = nullptr; R* dz = nullptr; R* r = nullptr; R* ir = nullptr; R* w = nullptr; R* dw = nullptr; R* omw = nullptr;
    R* nC = nullptr; R* nH = nullptr;
    // connectivity map: entries per atom and their hash table
    int map_cap = 0, map_hbits = 0;
    int* map_cnt = nullptr; R* map_wt = nullptr; int* map_path = nullptr;
    unsigned long long* map_ht = nullptr;     // 2^map_hbits slots per atom
    // FP32 copy of the short-list geometry for the b* screen (FP64 only)
    float* s_dx = nullptr; float* s_dy = nullptr; float* s_dz = nullptr; float* s_r = nullptr; float* s_ir = nullptr;
    float* s_w = nullptr; float* s_nC = nullptr; float* s_nH = nullptr;
};

// everything the compute kernels read, passed by value
template <class R> struct StepArgs {
    int n;
    const DevParams<R>* P;
    const DevParams<dd>* Pdd;              // AIREBO_DF64: the parameters in double-float (torsion), null otherwise
    Graph<R> G;
    int* g_cnt; int* g_nj; int* g_nimg;
    R* g_dx; R* g_dy; R* g_dz; R* g_r; R* g_ir; R* g_w; R* g_dw; R* g_omw; R* g_nC; R* g_nH;
    PathMap<R> M;
    const double* pos;
    float4* posf;                          // FP32 copy of the positions (written by the short-list kernel)
    float4* pq_lo;                         // split positions: the lo parts (posf holds the hi parts)
    const float4* Lhl;                     // per system: box edges split as hi + lo (2 float4)
    unsigned long long* fix;               // double-float LJ: fixed-point force sums (3 x n), null otherwise
    double L[3];
    const int2* lj; const int* lj_cnt; int lj_cap;
    const int2* im; const int* im_cnt; int im_cap;
    int2* bonds; int* nbonds; int bond_cap;   // C-H bonds from the carbon, from the front
    int* nhhbonds;                            // H-H bonds i<j, in the same array from its far end
    int2* ccbonds; int* nccbonds;             // C-C bonds i<j, same capacity
    int4* bq; int* nbq; int bq_cap;
    int* bq2; int* nbq2;                   // b* pairs left to the full-precision pass, by species pair (3 x bq_cap)
    int4* pq; int* npq;                    // LJ pairs along a path for k_lj_path (FP64 arithmetic; bq_cap)
    // b* screen (FP64): an FP32 b* with a rigorous error bound decides S_b
    // where the whole bound lies outside the transition
    bool screen;
    const DevParams<ef>* Pef;              // the parameters with their FP32 rounding errors
    Graph<float> G32;                      // reads the s_* arrays below
    float* s_dx; float* s_dy; float* s_dz; float* s_r; float* s_ir; float* s_w; float* s_nC; float* s_nH;
    int* lj_next;                          // work counter of the LJ kernel's warps
    int lj_chunk;                          // atoms a warp takes at a time (tuned)
    int bond_waves;                        // waves of resident blocks of the REBO and torsion kernels (tuned)
    int bstar_waves;                       // waves of resident blocks of the b* kernels (tuned)
    const int* sys;                        // batched systems: system of each atom (null: one system, box L)
    const double* Lsys;                    // batched systems: box of each system (3 per system)
    double* eatom;                         // nullable: per-atom energies (each term split evenly between its i and j)
    double* f;
    double* acc;          // E_rebo, E_lj, E_tors, W[6]
    unsigned long long* counters;   // [8]
    int* err;             // [4]: max short-list count, map overflow, queue overflow, nonfinite
    bool virial;
    bool rebo, lj_on, torsion;
    double* pgrad;        // nullable: dE/d eps[3], dE/d sigma[3] of the inter-molecular term
    const double* jv;     // nullable: a direction v (3 x n) for the parameter derivatives of the forces
    double* jout;         // with jv: v . dF/d eps[3], v . dF/d sigma[3]
};

enum { ERR_SHORT = 0, ERR_MAP = 1, ERR_QUEUE = 2, ERR_NONFINITE = 3, ERR_DF = 4 };
// bits of err[ERR_NONFINITE] and err[ERR_DF]: each condition has its own bit,
// so that one evaluation can report several
enum { NONFINITE_POS = 1, NONFINITE_OVERLAP = 2 };
enum { DF_RANGE = 1, DF_FORCE = 2 };
enum { CNT_BONDS = 0, CNT_BSTAR = 1, CNT_DSB = 2, CNT_LJ = 3, CNT_MAP = 4, CNT_BSTAR_FULL = 7 };

// The FP64 evaluation of b* differs from the exact value of its formula by
// its own rounding (of order 1e-14 for these magnitudes); the screen's bound
// is against the exact value, so a decision needs this much more room (an
// FP32 constant of at least 1e-9).
constexpr float BSTAR_SCREEN_SLACK = 1.1e-9f;

// launchers, one instantiation per precision (kernels_f64.cu, kernels_f32.cu)
// ev (nullable): 7 events recorded before each of the 6 stages and after the last
template <class R> void launch_compute(const StepArgs<R>& a, cudaStream_t s, int num_sms, cudaEvent_t* ev);
// check of the b* screen's error bound on every queued pair (kernels_f64.cu)
void launch_bstar_bound_check(const StepArgs<double>& a, double* out, cudaStream_t s, int num_sms);

// neighbour build (neighbor.cu)
struct NeighborArgs {
    int n;
    const double* pos;
    const int8_t* type;
    double L[3];
    int nc[3], reach[3];
    double cell_w[3];
    float lj_rc[3];       // (3 sigma + skin + margin) per pair, squared below
    float im_rc[3];       // (Dmax + skin + margin)
    bool with_lj;         // build the LJ half list (off for REBO-only runs)
    int* cell_of; int* cell_count; int* cell_start; int* cell_fill;
    float4* spos; char4* swrap;
    int2* lj; int* lj_cnt; int lj_cap;
    int2* im; int* im_cnt; int im_cap;
    int* err;             // [0] max lj count, [1] max im count, [2] nonfinite / out of range, [3] bad type
    double* xref;         // copy of positions at the build (rebuild trigger)
    // batched systems (all null for one system): per atom its system; per
    // system its box, cell grid (cells, stencil reach, cell width) and first cell
    const int* sys;
    const double* Lsys;
    const int* snc;
    const int* sreach;
    const double* scw;
    const int* scell0;
    // device-decided rebuild (the asynchronous MD step): when set, every
    // kernel of the build returns at once unless *gate is nonzero
    const int* gate;
};
void launch_neighbor(NeighborArgs& a, cudaStream_t s, int ncell);
// the same build behind a.gate, with the cell counts cleared and the
// reference positions copied by gated kernels too (no host work at all)
void launch_neighbor_gated(NeighborArgs& a, cudaStream_t s, int ncell);
// *gate = max displacement^2 > half2, and the device build counter counts it
void launch_rebuild_decide(const unsigned long long* maxd2_bits, double half2, int* gate, long long* builds,
                           cudaStream_t s);
// per-system sums of per-atom energies (one block per system)
void launch_system_energy(const double* eatom, const long long* offsets, int nsys, double* out, cudaStream_t s);

// NVE helpers (neighbor.cu)
void launch_nve_half(double* pos, double* vel, const double* f, const int8_t* type, int n, double dt,
                     bool drift, const double* xref, unsigned long long* maxdisp2_bits, double* ke, cudaStream_t s);
double alu_peak(int fp64);
int math_check(long long* out4);
int dd_check(double* out8);
void launch_max_disp(const double* pos, const double* xref, int n, unsigned long long* maxdisp2_bits, cudaStream_t s);

}  // namespace airebo
