// Host side of libairebo: the C ABI of include/airebo.h.
//
// Parses the parameter text, builds the power-basis coefficients of every
// spline (quintic per interval for g, bicubic for P, tricubic for pi^rc and
// T -- the Hermite interpolants of the knot data), owns every device buffer,
// and sequences the kernels of a step on the handle's stream.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>
#include <algorithm>

#include "../../include/airebo.h"
#include "internal.h"

using namespace airebo;

namespace {

// ------------------------------------------------------------------ parameters
struct HostParams {
    std::map<std::string, std::vector<double>> v;
    bool get(const char* k, size_t n, std::vector<double>& out, std::string& err) const {
        auto it = v.find(k);
        if (it == v.end() || it->second.size() != n) {
            err = std::string("parameter ") + k + " missing or of wrong size";
            return false;
        }
        out = it->second;
        return true;
    }
};

bool parse_text(const char* text, HostParams& hp, std::string& err) {
    std::istringstream in(text);
    std::string line;
    int nlines = 0;
    while (std::getline(in, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream ls(line);
        std::string name;
        long long n;
        if (!(ls >> name >> n) || n < 0 || n > 100000) { err = "bad parameter line: " + line.substr(0, 60); return false; }
        std::vector<double> vals((size_t)n);
        for (long long k = 0; k < n; k++)
            if (!(ls >> vals[k])) { err = "too few values for " + name; return false; }
        hp.v[name] = vals;
        nlines++;
    }
    if (!nlines) { err = "empty parameter text"; return false; }
    return true;
}

// cubic Hermite basis on [0,1] in powers of t: [kind][end][power];
// kind 0 = value basis, 1 = slope basis; end 0 = t=0, 1 = t=1
const double HB[2][2][4] = {
    {{1, 0, -3, 2}, {0, 0, 3, -2}},
    {{0, 1, -2, 1}, {0, 0, -1, 1}},
};

// knot data (5 x 5 grid, f fx fy fxy) -> 16 cells x 16 coefficients a[p*4+q]
void bicubic_coeffs(const std::vector<double>& d, double* out) {
    const int comp[2][2] = {{0, 2}, {1, 3}};   // [dx][dy]
    for (int ix = 0; ix < 4; ix++)
        for (int iy = 0; iy < 4; iy++) {
            double* a = out + (ix * 4 + iy) * 16;
            for (int k = 0; k < 16; k++) a[k] = 0;
            for (int ex = 0; ex < 2; ex++)
                for (int ey = 0; ey < 2; ey++)
                    for (int dx = 0; dx < 2; dx++)
                        for (int dy = 0; dy < 2; dy++) {
                            double val = d[((ix + ex) * 5 + (iy + ey)) * 4 + comp[dx][dy]];
                            if (val == 0.0) continue;
                            for (int p = 0; p < 4; p++)
                                for (int q = 0; q < 4; q++)
                                    a[p * 4 + q] += val * HB[dx][ex][p] * HB[dy][ey][q];
                        }
        }
}

// knot data (5 x 5 x 9 grid, f fx fy fz fxy fxz fyz fxyz) -> 128 cells x 64 a[(p*4+q)*4+r]
void tricubic_coeffs(const std::vector<double>& d, double* out, unsigned char* nz) {
    int comp[2][2][2];
    comp[0][0][0] = 0; comp[1][0][0] = 1; comp[0][1][0] = 2; comp[0][0][1] = 3;
    comp[1][1][0] = 4; comp[1][0][1] = 5; comp[0][1][1] = 6; comp[1][1][1] = 7;
    for (int ix = 0; ix < 4; ix++)
        for (int iy = 0; iy < 4; iy++)
            for (int iz = 0; iz < 8; iz++) {
                int cell = (ix * 4 + iy) * 8 + iz;
                double* a = out + cell * 64;
                for (int k = 0; k < 64; k++) a[k] = 0;
                bool any = false;
                for (int ex = 0; ex < 2; ex++)
                    for (int ey = 0; ey < 2; ey++)
                        for (int ez = 0; ez < 2; ez++)
                            for (int dx = 0; dx < 2; dx++)
                                for (int dy = 0; dy < 2; dy++)
                                    for (int dz = 0; dz < 2; dz++) {
                                        double val = d[(((ix + ex) * 5 + (iy + ey)) * 9 + (iz + ez)) * 8 + comp[dx][dy][dz]];
                                        if (val == 0.0) continue;
                                        any = true;
                                        for (int p = 0; p < 4; p++)
                                            for (int q = 0; q < 4; q++)
                                                for (int r = 0; r < 4; r++)
                                                    a[(p * 4 + q) * 4 + r] += val * HB[dx][ex][p] * HB[dy][ey][q] * HB[dz][ez][r];
                                    }
                if (nz) nz[cell] = any ? 1 : 0;
            }
}

// quintic Hermite basis in powers of t: value, slope, curvature at t=0, then curvature, slope, value at t=1
const double QB[6][6] = {
    {1, 0, 0, -10, 15, -6},
    {0, 1, 0, -6, 8, -3},
    {0, 0, 0.5, -1.5, 1.5, -0.5},
    {0, 0, 0, 0.5, -1, 0.5},
    {0, 0, 0, -4, 7, -3},
    {0, 0, 0, 10, -15, 6},
};

template <class R>
bool quintic_coeffs(const std::vector<double>& kn, const std::vector<double>& d, Quintic<R>& q, std::string& err) {
    int n = (int)kn.size() - 1;
    if (n < 1 || n > 5 || d.size() != kn.size() * 3) { err = "bad angular spline"; return false; }
    q.n = n;
    for (int m = 0; m <= n; m++) q.k[m] = (R)kn[m];
    for (int m = n + 1; m < 6; m++) q.k[m] = (R)kn[n];
    for (int m = 0; m < 5; m++) {
        q.invh[m] = 0;
        for (int p = 0; p < 6; p++) q.a[m][p] = 0;
        for (int p = 0; p < 5; p++) q.da[m][p] = 0;
    }
    for (int m = 0; m < n; m++) {
        double h = kn[m + 1] - kn[m];
        if (!(h > 0)) { err = "angular spline knots not increasing"; return false; }
        q.invh[m] = (R)(1.0 / h);
        double w[6] = {d[3 * m], h * d[3 * m + 1], h * h * d[3 * m + 2],
                       h * h * d[3 * (m + 1) + 2], h * d[3 * (m + 1) + 1], d[3 * (m + 1)]};
        double s[6];
        for (int p = 0; p < 6; p++) {
            s[p] = 0;
            for (int b = 0; b < 6; b++) s[p] += w[b] * QB[b][p];
            q.a[m][p] = (R)s[p];
        }
        for (int p = 0; p < 5; p++) q.da[m][p] = (R)((p + 1) * s[p + 1] / h);
    }
    return true;
}

// Transposes of the three coefficient builders above: given dE/d(coefficient),
// accumulate dE/d(knot datum).  The builders are linear in the knot data, so
// these are exact.
void bicubic_coeffs_adjoint(const double* g, double* out) {
    const int comp[2][2] = {{0, 2}, {1, 3}};
    for (int ix = 0; ix < 4; ix++)
        for (int iy = 0; iy < 4; iy++) {
            const double* a = g + (ix * 4 + iy) * 16;
            for (int ex = 0; ex < 2; ex++)
                for (int ey = 0; ey < 2; ey++)
                    for (int dx = 0; dx < 2; dx++)
                        for (int dy = 0; dy < 2; dy++) {
                            double s = 0;
                            for (int p = 0; p < 4; p++)
                                for (int q = 0; q < 4; q++) s += a[p * 4 + q] * HB[dx][ex][p] * HB[dy][ey][q];
                            out[((ix + ex) * 5 + (iy + ey)) * 4 + comp[dx][dy]] += s;
                        }
        }
}

void tricubic_coeffs_adjoint(const double* g, double* out) {
    int comp[2][2][2];
    comp[0][0][0] = 0; comp[1][0][0] = 1; comp[0][1][0] = 2; comp[0][0][1] = 3;
    comp[1][1][0] = 4; comp[1][0][1] = 5; comp[0][1][1] = 6; comp[1][1][1] = 7;
    for (int ix = 0; ix < 4; ix++)
        for (int iy = 0; iy < 4; iy++)
            for (int iz = 0; iz < 8; iz++) {
                const double* a = g + ((ix * 4 + iy) * 8 + iz) * 64;
                for (int ex = 0; ex < 2; ex++)
                    for (int ey = 0; ey < 2; ey++)
                        for (int ez = 0; ez < 2; ez++)
                            for (int dx = 0; dx < 2; dx++)
                                for (int dy = 0; dy < 2; dy++)
                                    for (int dz = 0; dz < 2; dz++) {
                                        double s = 0;
                                        for (int p = 0; p < 4; p++)
                                            for (int q = 0; q < 4; q++) {
                                                double hpq = HB[dx][ex][p] * HB[dy][ey][q];
                                                for (int r = 0; r < 4; r++)
                                                    s += a[(p * 4 + q) * 4 + r] * hpq * HB[dz][ez][r];
                                            }
                                        out[(((ix + ex) * 5 + (iy + ey)) * 9 + (iz + ez)) * 8 + comp[dx][dy][dz]] += s;
                                    }
            }
}

// g: [interval m][power p]; out: (value, slope, curvature) per knot
void quintic_coeffs_adjoint(const std::vector<double>& kn, const double* g, double* out) {
    int n = (int)kn.size() - 1;
    for (int m = 0; m < n; m++) {
        double h = kn[m + 1] - kn[m];
        double gw[6];
        for (int b = 0; b < 6; b++) {
            gw[b] = 0;
            for (int p = 0; p < 6; p++) gw[b] += QB[b][p] * g[m * 6 + p];
        }
        out[3 * m] += gw[0];
        out[3 * m + 1] += h * gw[1];
        out[3 * m + 2] += h * h * gw[2];
        out[3 * (m + 1) + 2] += h * h * gw[3];
        out[3 * (m + 1) + 1] += h * gw[4];
        out[3 * (m + 1)] += gw[5];
    }
}

struct Scalars {
    double Dmin[3], Dmax[3], Q[3], alpha[3], A[3], B[3][3], beta[3][3], rho[3];
    double lam, gN[2], Fx[2], guard[2], sigma[3], eps[3], ljcut, ljsw, Sr[2], bmin[3], bmax[3], rstar[3], teps[3];
    int kind = 0;
    double meps[3] = {0, 0, 0}, malpha[3] = {0, 0, 0}, mre[3] = {0, 0, 0};
    std::vector<double> gC1k, gC1d, gC2k, gC2d, gHk, gHd;
    std::vector<double> P[3], F[3], T;
};

bool load_scalars(const HostParams& hp, Scalars& s, std::string& err) {
    std::vector<double> t;
    auto g3 = [&](const char* k, double* dst) { if (!hp.get(k, 3, t, err)) return false; for (int i = 0; i < 3; i++) dst[i] = t[i]; return true; };
    double b1[3], b2[3], b3[3], e1[3], e2[3], e3[3];
    if (!(g3("Dmin", s.Dmin) && g3("Dmax", s.Dmax) && g3("Q", s.Q) && g3("alpha", s.alpha) && g3("A", s.A) &&
          g3("B1", b1) && g3("B2", b2) && g3("B3", b3) && g3("beta1", e1) && g3("beta2", e2) && g3("beta3", e3) &&
          g3("rho", s.rho) && g3("lj.sigma", s.sigma) && g3("lj.epsilon", s.eps) && g3("bstar.bmin", s.bmin) &&
          g3("bstar.bmax", s.bmax) && g3("bstar.rstar", s.rstar) && g3("tors.epsilon", s.teps)))
        return false;
    for (int i = 0; i < 3; i++) {
        s.B[i][0] = b1[i]; s.B[i][1] = b2[i]; s.B[i][2] = b3[i];
        s.beta[i][0] = e1[i]; s.beta[i][1] = e2[i]; s.beta[i][2] = e3[i];
    }
    auto g1 = [&](const char* k, double& dst) { if (!hp.get(k, 1, t, err)) return false; dst = t[0]; return true; };
    auto g2 = [&](const char* k, double* dst) { if (!hp.get(k, 2, t, err)) return false; dst[0] = t[0]; dst[1] = t[1]; return true; };
    if (!(g1("lambda_coef", s.lam) && g2("gC_Nswitch", s.gN) && g2("Fconj_x", s.Fx) && g2("dihedral_guard", s.guard) &&
          g1("lj.cut", s.ljcut) && g1("lj.switch_start", s.ljsw) && g2("lj.Sr_range", s.Sr)))
        return false;
    if (!(hp.get("gC1.knots", 6, s.gC1k, err) && hp.get("gC1.data", 18, s.gC1d, err) &&
          hp.get("gC2.knots", 6, s.gC2k, err) && hp.get("gC2.data", 18, s.gC2d, err) &&
          hp.get("gH.knots", 4, s.gHk, err) && hp.get("gH.data", 12, s.gHd, err) &&
          hp.get("P.CC", 100, s.P[0], err) && hp.get("P.CH", 100, s.P[1], err) && hp.get("P.HC", 100, s.P[2], err) &&
          hp.get("piRC.CC", 1800, s.F[0], err) && hp.get("piRC.CH", 1800, s.F[1], err) &&
          hp.get("piRC.HH", 1800, s.F[2], err) && hp.get("Tij.CC", 1800, s.T, err)))
        return false;
    {
        auto it = hp.v.find("inter.kind");
        s.kind = (it != hp.v.end() && it->second.size() == 1) ? (int)it->second[0] : 0;
        if (s.kind != 0 && s.kind != 1) { err = "inter.kind must be 0 (Lennard-Jones) or 1 (Morse)"; return false; }
        if (s.kind == 1 && !(g3("morse.epsilon", s.meps) && g3("morse.alpha", s.malpha) && g3("morse.re", s.mre)))
            return false;
    }
    for (int p = 0; p < 3; p++) {
        if (!(s.Dmax[p] > s.Dmin[p] && s.Dmin[p] > 0)) { err = "Dmax must exceed Dmin > 0"; return false; }
        if (!(s.sigma[p] > 0 && s.bmax[p] > s.bmin[p] && s.rstar[p] > 0)) { err = "bad LJ/b* parameter"; return false; }
    }
    if (!(s.ljcut > s.ljsw && s.ljsw > 0 && s.Sr[1] > s.Sr[0] && s.gN[1] > s.gN[0] && s.Fx[1] > s.Fx[0] && s.guard[1] > 0)) {
        err = "bad switch parameter";
        return false;
    }
    return true;
}

// the device tables of one precision: spline coefficients, then knot data
constexpr int PKNOT_OFF = 3 * 256 + 4 * NTRI_CELLS * 64;
constexpr int TABLES_LEN = PKNOT_OFF + 3 * 25 * 3 + 4 * 225 * 4;

template <class R>
bool fill_params(const Scalars& s, DevParams<R>& P, std::vector<R>& tables, std::vector<unsigned char>& Tnz, std::string& err) {
    for (int p = 0; p < 3; p++) {
        P.Dmin[p] = (R)s.Dmin[p]; P.Dmax[p] = (R)s.Dmax[p]; P.Dinv[p] = (R)(1.0 / (s.Dmax[p] - s.Dmin[p]));
        P.Q[p] = (R)s.Q[p]; P.alpha[p] = (R)s.alpha[p]; P.A[p] = (R)s.A[p];
        int nb = 0;
        for (int m = 0; m < 3; m++) {
            P.B[p][m] = 0; P.beta[p][m] = 0;
            if (s.B[p][m] != 0.0) { P.B[p][nb] = (R)s.B[p][m]; P.beta[p][nb] = (R)s.beta[p][m]; nb++; }
        }
        P.nB[p] = nb;
        double sg = s.sigma[p];
        P.sigma[p] = (R)sg;
        P.sig2[p] = (R)(sg * sg);
        P.eps4[p] = (R)(4.0 * s.eps[p]);
        P.rc2[p] = (R)(s.ljcut * sg * s.ljcut * sg);
        P.swlo[p] = (R)(s.ljsw * sg);
        P.swlo2[p] = (R)(s.ljsw * sg * s.ljsw * sg);
        P.swinv[p] = (R)(1.0 / ((s.ljcut - s.ljsw) * sg));
        P.Srlo[p] = (R)(s.Sr[0] * sg);
        P.Srhi[p] = (R)(s.Sr[1] * sg);
        P.Srhi2[p] = (R)(s.Sr[1] * sg * s.Sr[1] * sg);
        P.Srinv[p] = (R)(1.0 / ((s.Sr[1] - s.Sr[0]) * sg));
        P.bmin[p] = (R)s.bmin[p];
        P.bmax[p] = (R)s.bmax[p];
        P.binv[p] = (R)(1.0 / (s.bmax[p] - s.bmin[p]));
        P.rstar[p] = (R)s.rstar[p];
        P.teps[p] = (R)s.teps[p];
        P.meps[p] = (R)s.meps[p];
        P.malpha[p] = (R)s.malpha[p];
        P.mre[p] = (R)s.mre[p];
    }
    P.kind = s.kind;
    P.rhoH[0] = (R)s.rho[1];   // H centre, C neighbour: rho_CH
    P.rhoH[1] = (R)s.rho[2];   // H centre, H neighbour: rho_HH
    P.lam = (R)s.lam;
    P.gN0 = (R)s.gN[0]; P.gNinv = (R)(1.0 / (s.gN[1] - s.gN[0]));
    P.Fx0 = (R)s.Fx[0]; P.Fxinv = (R)(1.0 / (s.Fx[1] - s.Fx[0]));
    P.guard0 = (R)s.guard[0]; P.guardinv = (R)(1.0 / s.guard[1]);
    double dm = std::max(s.Dmax[0], std::max(s.Dmax[1], s.Dmax[2]));
    P.rpath2 = (R)(9.0 * dm * dm * (1.0 + 1e-6));
    if (!quintic_coeffs<R>(s.gC1k, s.gC1d, P.gC1, err) || !quintic_coeffs<R>(s.gC2k, s.gC2d, P.gC2, err) ||
        !quintic_coeffs<R>(s.gHk, s.gHd, P.gH, err))
        return false;
    // tables: P (3 x 256), pi^rc (3 x 8192), T (8192) coefficients, then the
    // knot data: P (3 x 25 x 3), pi^rc (3 x 225 x 4), T (225 x 4)
    std::vector<double> buf(TABLES_LEN);
    for (int t = 0; t < 3; t++) bicubic_coeffs(s.P[t], buf.data() + t * 256);
    for (int t = 0; t < 3; t++) tricubic_coeffs(s.F[t], buf.data() + 3 * 256 + t * NTRI_CELLS * 64, nullptr);
    Tnz.assign(NTRI_CELLS, 0);
    tricubic_coeffs(s.T, buf.data() + 3 * 256 + 3 * NTRI_CELLS * 64, Tnz.data());
    double* kp = buf.data() + PKNOT_OFF;
    for (int t = 0; t < 3; t++)
        for (int k = 0; k < 25; k++)
            for (int c = 0; c < 3; c++) *kp++ = s.P[t][k * 4 + c];          // f, fx, fy
    for (int t = 0; t < 4; t++)                                            // pi^rc CC, CH, HH, then T_CC
        for (int k = 0; k < 225; k++)
            for (int c = 0; c < 4; c++) *kp++ = (t < 3 ? s.F[t] : s.T)[k * 8 + c];   // f, fx, fy, fz
    tables.resize(buf.size());
    for (size_t k = 0; k < buf.size(); k++) tables[k] = (R)buf[k];
    return true;
}

}  // namespace

// ------------------------------------------------------------------ handle
template <class R> struct Precision {
    DevParams<R> hp;                 // host copy, table pointers already device pointers
    StepBuffers<R> b;
    std::vector<R> tables;
    std::vector<unsigned char> Tnz;
};

struct airebo_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 1;
    airebo_options opt{};
    std::string err;
    Scalars sc;
    Precision<double> p64;
    Precision<float> p32;
    Precision<dd> pdd;        // AIREBO_DF64: the parameters in double-float (torsion kernel)
    Precision<ef> pef;        // the b* screen: the parameters in FP32 with their rounding errors
    // system
    int n = 0, n_alloc = 0;
    double L[3] = {0, 0, 0};
    int8_t* types = nullptr;
    bool built = false;
    // cells
    int nc[3] = {0, 0, 0}, reach[3] = {0, 0, 0}, ncell_alloc = 0;
    double cell_w[3] = {0, 0, 0};
    int *cell_of = nullptr, *cell_count = nullptr, *cell_start = nullptr, *cell_fill = nullptr;
    float4* spos = nullptr;
    float4* posf = nullptr;              // FP32 positions of the current step (LJ pair tests)
    float4* pq_lo = nullptr;             // split positions (lo parts) and fixed-point LJ force sums
    unsigned long long* fix = nullptr;
    char4* swrap = nullptr;
    // lists
    int2* lj = nullptr; int* lj_cnt = nullptr; int lj_cap = 0; size_t lj_alloc = 0;
    int2* im = nullptr; int* im_cnt = nullptr; int im_cap = 32; size_t im_alloc = 0;
    double* xref = nullptr;
    // step scratch
    int2* bonds = nullptr; int2* ccbonds = nullptr; int bond_cap = 0;
    int4* bq = nullptr; int bq_cap = 0;
    int* bq2 = nullptr;
    int4* pq = nullptr;             // LJ pairs along a path (0 < C_ij < 1), FP64 arithmetic
    int* counts = nullptr;               // [0] non-C-C bonds [2] C-C bonds [3] b* reverse queue [4..6] b* queue per species pair [7] LJ work counter
    double* acc = nullptr;               // 9 doubles
    unsigned long long* counters = nullptr;   // 8
    int* derr = nullptr;                 // 8 ints
    int stride = 8;                      // REBO slots per atom (grows to MAXN)
    // launch shapes (airebo_autotune); the defaults are the tuned shapes of the
    // 1M-atom PE in FP64 (grids of one b* pair or bond per thread at that size)
    int lj_chunk = 2, bond_waves = 16, bstar_waves = 16;
    // batched systems (nsys = 0: one system with box L)
    int nsys = 0;
    std::vector<double> Lsys_h;
    std::vector<long long> off_h;
    int *d_sys = nullptr, *d_snc = nullptr, *d_sreach = nullptr, *d_scell0 = nullptr;
    double *d_Lsys = nullptr, *d_scw = nullptr;
    float4* d_Lhl = nullptr;             // per system: box edges split as hi (2^-12 grid) + lo
    long long* d_off = nullptr;
    double* eatom = nullptr;
    int eatom_n = 0;
    // captured compute
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    unsigned long long* maxd2 = nullptr;
    double* ke = nullptr;
    // asynchronous MD step: the device's rebuild decision, its count of the
    // builds it ran, the sticky error flags of those builds (read and cleared
    // by airebo_check), and the arguments of the last synchronous build
    int* gate = nullptr;
    long long* d_builds = nullptr;
    int* nerr = nullptr;
    NeighborArgs nargs{};
    int nargs_ncell = 0;
    bool nargs_ok = false;
    double* pg = nullptr;                // parameter gradients (6)
    double* kg = nullptr;                // spline-coefficient gradients (KG_N)
    // pinned mirrors
    int* h_err = nullptr;
    unsigned long long* h_u64 = nullptr;
    double* h_acc = nullptr;
    // host-API staging
    double *hpos = nullptr, *hvel = nullptr, *hforce = nullptr, *he4 = nullptr, *hw6 = nullptr;
    int host_n = -1;
    long long rebuilds = 0;
    // per-kernel timing
    bool timing = false;
    cudaEvent_t ev[12] = {};             // 0..7 around the compute kernels, 8..11 neighbour build and NVE
    double kt_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    long long kt_n[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

airebo_status fail(airebo_handle h, airebo_status st, const std::string& msg) {
    if (h) h->err = msg;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(h, AIREBO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T> cudaError_t realloc_dev(T*& p, size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)&p, sizeof(T) * count);
}

template <class R> airebo_status upload_params(airebo_handle h, Precision<R>& pr) {
    std::string e;
    if (!fill_params<R>(h->sc, pr.hp, pr.tables, pr.Tnz, e)) return fail(h, AIREBO_ERR_ARG, e);
    CK(realloc_dev(pr.b.tables, pr.tables.size()));
    CK(realloc_dev(pr.b.Tnz, pr.Tnz.size()));
    CK(realloc_dev(pr.b.P, 1));
    CK(cudaMemcpy(pr.b.tables, pr.tables.data(), sizeof(R) * pr.tables.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pr.b.Tnz, pr.Tnz.data(), pr.Tnz.size(), cudaMemcpyHostToDevice));
    pr.hp.Ptab = pr.b.tables;
    pr.hp.Ftab = pr.b.tables + 3 * 256;
    pr.hp.Ttab = pr.b.tables + 3 * 256 + 3 * NTRI_CELLS * 64;
    pr.hp.Tnz = pr.b.Tnz;
    pr.hp.Pknot = pr.b.tables + PKNOT_OFF;
    pr.hp.Fknot = pr.hp.Pknot + 3 * 25 * 3;
    pr.hp.Tknot = pr.hp.Fknot + 3 * 225 * 4;
    pr.hp.kg = nullptr;
    CK(cudaMemcpy(pr.b.P, &pr.hp, sizeof(DevParams<R>), cudaMemcpyHostToDevice));
    return AIREBO_OK;
}

// the FP32 b* screen of the FP64 path (see k_bstar)
bool screen_on(airebo_handle h);

// the connectivity-map entries (map_cap per atom) and their hash tables (a
// power of two of at least twice as many slots)
template <class R> airebo_status alloc_map(airebo_handle h, StepBuffers<R>& b, int n) {
    if (b.map_cap > (1 << MAP_IDX_BITS)) return fail(h, AIREBO_ERR_CAPACITY, "connectivity map beyond 4096 entries per atom");
    b.map_hbits = 1;
    while ((1 << b.map_hbits) < 2 * b.map_cap) b.map_hbits++;
    size_t mm = (size_t)n * b.map_cap;
    CK(realloc_dev(b.map_wt, mm)); CK(realloc_dev(b.map_path, mm));
    CK(realloc_dev(b.map_ht, (size_t)n << b.map_hbits));
    return AIREBO_OK;
}

template <class R> airebo_status alloc_step(airebo_handle h, Precision<R>& pr, int n) {
    StepBuffers<R>& b = pr.b;
    size_t m = (size_t)n * h->stride;
    CK(realloc_dev(b.cnt, n)); CK(realloc_dev(b.nj, m)); CK(realloc_dev(b.nimg, m));
    CK(realloc_dev(b.dx, m)); CK(realloc_dev(b.dy, m)); CK(realloc_dev(b.dz, m));
    CK(realloc_dev(b.r, m)); CK(realloc_dev(b.ir, m)); CK(realloc_dev(b.w, m)); CK(realloc_dev(b.dw, m)); CK(realloc_dev(b.omw, m));
    CK(realloc_dev(b.nC, n)); CK(realloc_dev(b.nH, n));
    if (b.map_cap == 0) b.map_cap = 32;
    CK(realloc_dev(b.map_cnt, n));
    airebo_status st = alloc_map<R>(h, b, n);
    if (st) return st;
    if (sizeof(R) == 8 && screen_on(h)) {
        CK(realloc_dev(b.s_dx, m)); CK(realloc_dev(b.s_dy, m)); CK(realloc_dev(b.s_dz, m));
        CK(realloc_dev(b.s_r, m)); CK(realloc_dev(b.s_ir, m)); CK(realloc_dev(b.s_w, m));
        CK(realloc_dev(b.s_nC, n)); CK(realloc_dev(b.s_nH, n));
    }
    return AIREBO_OK;
}

template <class R> airebo_status grow_map(airebo_handle h, Precision<R>& pr, int need) {
    StepBuffers<R>& b = pr.b;
    b.map_cap = std::max(need + 8, b.map_cap * 2);
    return alloc_map<R>(h, b, h->n_alloc);
}

template <class R> void free_prec(Precision<R>& pr) {
    StepBuffers<R>& b = pr.b;
    void* ps[] = {b.P, b.Pkg, b.tables, b.Tnz, b.cnt, b.nj, b.nimg, b.dx, b.dy, b.dz, b.r, b.ir, b.w, b.dw, b.omw, b.nC, b.nH,
                  b.map_cnt, b.map_wt, b.map_path, b.map_ht,
                  b.s_dx, b.s_dy, b.s_dz, b.s_r, b.s_ir, b.s_w, b.s_nC, b.s_nH};
    for (void* p : ps) if (p) cudaFree(p);
    b = StepBuffers<R>();
}

double max3(const double* v) { return std::max(v[0], std::max(v[1], v[2])); }

// cells at least 1/CELL_DIV of the long cut-off wide (a 5 x 5 x 5 stencil for
// 2): the stencil then covers 15.6 instead of 27 cut-off cubes (measured on the
// 1M-atom PE: 9.0 -> 6.4 ms per list build; 3 gives no further gain)
constexpr int CELL_DIV = 2;

bool screen_on(airebo_handle h) {
    return h->opt.precision != AIREBO_MIXED && h->opt.bstar_screen != 0 && h->opt.enable_lj != 0;
}

// the parameter sets of the handle's precision: its own, the FP32 one of the
// b* screen, and for AIREBO_DF64 the double-float one of the torsion kernel
airebo_status upload_own_params(airebo_handle h) {
    airebo_status st = h->opt.precision == AIREBO_MIXED ? upload_params<float>(h, h->p32) : upload_params<double>(h, h->p64);
    if (!st && screen_on(h)) st = upload_params<ef>(h, h->pef);
    if (!st && h->opt.precision == AIREBO_DF64) st = upload_params<dd>(h, h->pdd);
    return st;
}

// the LJ kernel on split positions with fixed-point force sums: double-float
// pair arithmetic (AIREBO_DF64) or FP32 pair arithmetic (AIREBO_MIXED);
// Lennard-Jones form only
bool df_on(airebo_handle h) {
    return h->opt.precision != AIREBO_FP64 && h->opt.enable_lj != 0 && h->sc.kind == 0;
}

airebo_status alloc_atoms(airebo_handle h, int n) {
    if (n <= h->n_alloc && h->n_alloc > 0) return AIREBO_OK;
    int na = std::max(n, 1);
    CK(realloc_dev(h->types, na));
    CK(realloc_dev(h->cell_of, na));
    CK(realloc_dev(h->spos, na));
    CK(realloc_dev(h->posf, na));
    if (h->opt.precision != AIREBO_FP64) {
        CK(realloc_dev(h->pq_lo, na));
        CK(realloc_dev(h->fix, 3 * (size_t)na));
    }
    CK(realloc_dev(h->swrap, na));
    CK(realloc_dev(h->lj_cnt, na));
    CK(realloc_dev(h->im_cnt, na));
    CK(realloc_dev(h->xref, 3 * (size_t)na));
    h->bond_cap = na * MAXN / 2 + 64;
    CK(realloc_dev(h->bonds, h->bond_cap));
    CK(realloc_dev(h->ccbonds, h->bond_cap));
    h->bq_cap = std::max(h->bq_cap, na * 4 + 1024);
    CK(realloc_dev(h->bq, 3 * (size_t)h->bq_cap));
    CK(realloc_dev(h->bq2, 3 * (size_t)h->bq_cap));
    CK(realloc_dev(h->pq, (size_t)h->bq_cap));
    h->n_alloc = na;
    airebo_status st = h->opt.precision == AIREBO_MIXED ? alloc_step<float>(h, h->p32, na) : alloc_step<double>(h, h->p64, na);
    if (st) return st;
    h->lj_alloc = 0;
    h->im_alloc = 0;
    return AIREBO_OK;
}

airebo_status ensure_lists(airebo_handle h) {
    size_t need_lj = (size_t)h->n_alloc * h->lj_cap, need_im = (size_t)h->n_alloc * h->im_cap;
    if (need_lj > h->lj_alloc) { CK(realloc_dev(h->lj, need_lj)); h->lj_alloc = need_lj; }
    if (need_im > h->im_alloc) { CK(realloc_dev(h->im, need_im)); h->im_alloc = need_im; }
    return AIREBO_OK;
}

airebo_status do_neighbor(airebo_handle h, const double* d_pos) {
    const Scalars& s = h->sc;
    h->nargs_ok = false;            // the saved build arguments may point at buffers about to change
    double rlj = 0, rim = 0;
    NeighborArgs a{};
    bool with_lj = h->opt.enable_lj != 0;
    for (int p = 0; p < 3; p++) {
        double ri = s.Dmax[p] + h->opt.skin;
        double rc = with_lj ? s.ljcut * s.sigma[p] + h->opt.skin : ri;   // REBO only: no long list
        rlj = std::max(rlj, rc);
        rim = std::max(rim, ri);
        a.lj_rc[p] = (float)(rc + 2e-3);
        a.im_rc[p] = (float)(ri + 2e-3);
    }
    a.with_lj = with_lj;
    rlj += 2e-3;
    int ncell = 1;
    double rho_max = 0;
    // without the long list the cut-off is the REBO one: half of it would make
    // cells of less than one atom, whose per-cell work outweighs the pruning
    int div = h->opt.enable_lj ? CELL_DIV : 1;
    if (h->nsys == 0) {
        for (int d = 0; d < 3; d++) {
            h->nc[d] = std::max(1, (int)std::floor(h->L[d] * div / rlj));
            h->cell_w[d] = h->L[d] / h->nc[d];
            h->reach[d] = (int)std::ceil(rlj / h->cell_w[d]);
            ncell *= h->nc[d];
        }
        rho_max = h->n / (h->L[0] * h->L[1] * h->L[2]);
    } else {
        // one cell grid per system, numbered consecutively
        std::vector<int> nc(3 * h->nsys), reach(3 * h->nsys), cell0(h->nsys + 1);
        std::vector<double> cw(3 * h->nsys);
        ncell = 0;
        for (int s = 0; s < h->nsys; s++) {
            int cs = 1;
            for (int d = 0; d < 3; d++) {
                double L = h->Lsys_h[3 * s + d];
                nc[3 * s + d] = std::max(1, (int)std::floor(L * div / rlj));
                cw[3 * s + d] = L / nc[3 * s + d];
                reach[3 * s + d] = (int)std::ceil(rlj / cw[3 * s + d]);
                cs *= nc[3 * s + d];
            }
            cell0[s] = ncell;
            ncell += cs;
            double vol = h->Lsys_h[3 * s] * h->Lsys_h[3 * s + 1] * h->Lsys_h[3 * s + 2];
            rho_max = std::max(rho_max, (h->off_h[s + 1] - h->off_h[s]) / vol);
        }
        cell0[h->nsys] = ncell;
        CK(cudaMemcpyAsync(h->d_snc, nc.data(), sizeof(int) * nc.size(), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_sreach, reach.data(), sizeof(int) * reach.size(), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_scw, cw.data(), sizeof(double) * cw.size(), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_scell0, cell0.data(), sizeof(int) * cell0.size(), cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (ncell > h->ncell_alloc) {
        CK(realloc_dev(h->cell_count, ncell));
        CK(realloc_dev(h->cell_start, ncell + 1));
        CK(realloc_dev(h->cell_fill, ncell));
        h->ncell_alloc = ncell;
    }
    if (!with_lj) h->lj_cap = 1;
    if (h->lj_cap == 0) {
        double est = 0.5 * 4.0 / 3.0 * M_PI * rlj * rlj * rlj * rho_max;
        h->lj_cap = h->opt.max_lj_nbrs > 0 ? h->opt.max_lj_nbrs : ((int)(1.2 * est + 32) + 31) / 32 * 32;
    }
    for (int attempt = 0; attempt < 4; attempt++) {
        airebo_status st = ensure_lists(h);
        if (st) return st;
        a.n = h->n; a.pos = d_pos; a.type = h->types;
        for (int d = 0; d < 3; d++) { a.L[d] = h->L[d]; a.nc[d] = h->nc[d]; a.reach[d] = h->reach[d]; a.cell_w[d] = h->cell_w[d]; }
        a.cell_of = h->cell_of; a.cell_count = h->cell_count; a.cell_start = h->cell_start; a.cell_fill = h->cell_fill;
        a.spos = h->spos; a.swrap = h->swrap;
        a.lj = h->lj; a.lj_cnt = h->lj_cnt; a.lj_cap = h->lj_cap;
        a.im = h->im; a.im_cnt = h->im_cnt; a.im_cap = h->im_cap;
        a.err = h->derr; a.xref = h->xref;
        a.sys = h->nsys ? h->d_sys : nullptr;
        a.Lsys = h->nsys ? h->d_Lsys : nullptr;
        a.snc = h->d_snc; a.sreach = h->d_sreach; a.scw = h->d_scw; a.scell0 = h->d_scell0;
        CK(cudaMemsetAsync(h->derr, 0, sizeof(int) * 8, h->stream));
        if (h->timing) CK(cudaEventRecord(h->ev[8], h->stream));
        launch_neighbor(a, h->stream, ncell);
        CK(cudaGetLastError());
        if (h->timing) CK(cudaEventRecord(h->ev[9], h->stream));
        CK(cudaMemcpyAsync(h->h_err, h->derr, sizeof(int) * 8, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (h->timing && h->n) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, h->ev[8], h->ev[9]));
            h->kt_ms[6] += ms;
            h->kt_n[6] += 1;
        }
        if (h->h_err[2] == 1) { h->built = false; return fail(h, AIREBO_ERR_NONFINITE, "non-finite position"); }
        if (h->h_err[2] == 2) return fail(h, AIREBO_ERR_ARG, "position more than 120 box lengths outside the box");
        if (h->h_err[3]) { h->built = false; return fail(h, AIREBO_ERR_ARG, "atom type other than 0 (C) or 1 (H)"); }
        bool again = false;
        if (h->h_err[0] > h->lj_cap) { h->lj_cap = ((int)(h->h_err[0] * 1.1) + 32) / 32 * 32; again = true; }
        if (h->h_err[1] > h->im_cap) { h->im_cap = ((int)(h->h_err[1] * 1.2) + 8); again = true; }
        if (!again) {
            if (h->n) CK(cudaMemcpyAsync(h->xref, d_pos, sizeof(double) * 3 * h->n, cudaMemcpyDeviceToDevice, h->stream));
            h->built = true;
            h->rebuilds++;
            h->nargs = a;
            h->nargs_ncell = ncell;
            h->nargs_ok = true;
            return AIREBO_OK;
        }
    }
    return fail(h, AIREBO_ERR_CAPACITY, "neighbour list capacity did not converge");
}

__global__ void k_finalize(const double* acc, double* e4, double* w6) {
    int t = threadIdx.x;
    if (e4 && t < 4) e4[t] = t == 0 ? acc[0] + acc[1] + acc[2] : acc[t - 1];
    if (w6 && t < 6) w6[t] = acc[3 + t];
}

// The status of the device error flags of the last evaluation (h->h_err):
// non-finite positions, overlapping atoms, and the range limits of the split
// positions and fixed-point sums of AIREBO_MIXED / AIREBO_DF64.  Every
// condition found is named in the message; the status is that of the first.
airebo_status device_errors(airebo_handle h) {
    int nf = h->h_err[ERR_NONFINITE], df = h->h_err[ERR_DF];
    if (!nf && !df) return AIREBO_OK;
    std::string msg;
    airebo_status st = AIREBO_OK;
    auto add = [&](airebo_status s2, const char* m) {
        if (!msg.empty()) msg += "; ";
        msg += m;
        if (st == AIREBO_OK) st = s2;
    };
    if (nf & NONFINITE_POS) add(AIREBO_ERR_NONFINITE, "non-finite position");
    if (nf & NONFINITE_OVERLAP) add(AIREBO_ERR_NONFINITE, "two atoms closer than 1e-6 A (overlapping atoms)");
    if (df & DF_RANGE) add(AIREBO_ERR_ARG, "AIREBO_DF64 and AIREBO_MIXED need every |coordinate| below 2000 A");
    if (df & DF_FORCE) add(AIREBO_ERR_NONFINITE, "an LJ pair force beyond the fixed-point range (1e6 eV/A)");
    return fail(h, st, msg);
}

template <class R> StepArgs<R> make_args(airebo_handle h, Precision<R>& pr, const double* d_pos, double* d_force, bool virial) {
    StepArgs<R> a{};
    StepBuffers<R>& b = pr.b;
    a.n = h->n;
    a.P = b.P;
    a.Pdd = h->opt.precision == AIREBO_DF64 ? h->pdd.b.P : nullptr;
    a.G.n = h->n; a.G.stride = h->stride; a.G.type = h->types; a.G.cnt = b.cnt; a.G.nj = b.nj; a.G.nimg = b.nimg;
    a.G.dx = b.dx; a.G.dy = b.dy; a.G.dz = b.dz; a.G.r = b.r; a.G.ir = b.ir; a.G.w = b.w; a.G.dw = b.dw; a.G.omw = b.omw; a.G.nC = b.nC; a.G.nH = b.nH;
    a.g_cnt = b.cnt; a.g_nj = b.nj; a.g_nimg = b.nimg; a.g_dx = b.dx; a.g_dy = b.dy; a.g_dz = b.dz;
    a.g_r = b.r; a.g_ir = b.ir; a.g_w = b.w; a.g_dw = b.dw; a.g_omw = b.omw; a.g_nC = b.nC; a.g_nH = b.nH;
    a.M.cap = b.map_cap; a.M.cnt = b.map_cnt; a.M.wt = b.map_wt; a.M.path = b.map_path;
    a.M.hbits = b.map_hbits; a.M.ht = b.map_ht;
    a.pos = d_pos;
    a.posf = h->posf;
    bool df = df_on(h);
    a.pq_lo = df ? h->pq_lo : nullptr;
    a.Lhl = h->d_Lhl;
    a.fix = df ? h->fix : nullptr;
    for (int d = 0; d < 3; d++) a.L[d] = h->L[d];
    a.lj = h->lj; a.lj_cnt = h->lj_cnt; a.lj_cap = h->lj_cap;
    a.im = h->im; a.im_cnt = h->im_cnt; a.im_cap = h->im_cap;
    a.bonds = h->bonds; a.nbonds = h->counts; a.bond_cap = h->bond_cap; a.nhhbonds = h->counts + 1;
    a.ccbonds = h->ccbonds; a.nccbonds = h->counts + 2;
    a.bq = h->bq; a.nbq = h->counts + 4; a.bq_cap = h->bq_cap;
    a.bq2 = h->bq2; a.nbq2 = h->counts + 8;
    a.pq = h->pq; a.npq = h->counts + 3;
    a.screen = false;
    a.Pef = nullptr;
    a.G32 = Graph<float>{};
    a.s_dx = a.s_dy = a.s_dz = a.s_r = a.s_ir = a.s_w = a.s_nC = a.s_nH = nullptr;
    if (sizeof(R) == 8 && screen_on(h) && b.s_dx) {
        a.screen = true;
        a.Pef = h->pef.b.P;
        a.s_dx = b.s_dx; a.s_dy = b.s_dy; a.s_dz = b.s_dz; a.s_r = b.s_r; a.s_ir = b.s_ir; a.s_w = b.s_w;
        a.s_nC = b.s_nC; a.s_nH = b.s_nH;
        a.G32.n = h->n; a.G32.stride = h->stride; a.G32.type = h->types; a.G32.cnt = b.cnt; a.G32.nj = b.nj;
        a.G32.nimg = b.nimg;
        a.G32.dx = b.s_dx; a.G32.dy = b.s_dy; a.G32.dz = b.s_dz; a.G32.r = b.s_r; a.G32.ir = b.s_ir; a.G32.w = b.s_w;
        a.G32.dw = nullptr; a.G32.omw = nullptr;        // the forward bond order reads neither
        a.G32.nC = b.s_nC; a.G32.nH = b.s_nH;
    }
    a.lj_next = h->counts + 7;
    a.lj_chunk = h->lj_chunk;
    a.bond_waves = h->bond_waves;
    a.bstar_waves = h->bstar_waves;
    a.f = d_force; a.acc = h->acc; a.counters = h->counters; a.err = h->derr;
    a.virial = virial;
    a.sys = h->nsys ? h->d_sys : nullptr;
    a.Lsys = h->nsys ? h->d_Lsys : nullptr;
    a.eatom = nullptr;
    a.pgrad = nullptr;
    a.jv = nullptr;
    a.jout = nullptr;
    a.rebo = h->opt.enable_rebo != 0;
    a.lj_on = h->opt.enable_lj != 0;
    a.torsion = h->opt.enable_torsion != 0;
    return a;
}

// One evaluation.  d_esys: per-system energies wanted (sums of the per-atom
// energies); d_eatom: per-atom energies wanted in the caller's buffer (also
// the source of d_esys then).  async: enqueue only (no host synchronisation,
// no regrowth; the capacity flags are read by airebo_check), as needed for
// graph capture.
template <class R>
airebo_status do_compute(airebo_handle h, Precision<R>& pr, const double* d_pos, double* d_force, double* d_e4,
                         double* d_w6, double* d_pgrad = nullptr, double* d_esys = nullptr, bool async = false,
                         double* d_kg = nullptr, double* d_eatom = nullptr, const double* d_jv = nullptr,
                         double* d_jout = nullptr) {
    for (int attempt = 0; attempt < 4; attempt++) {
        cudaStream_t s = h->stream;
        if (h->n) CK(cudaMemsetAsync(d_force, 0, sizeof(double) * 3 * h->n, s));
        CK(cudaMemsetAsync(h->acc, 0, sizeof(double) * 9, s));
        CK(cudaMemsetAsync(h->counters, 0, sizeof(unsigned long long) * 8, s));
        CK(cudaMemsetAsync(h->counts, 0, sizeof(int) * 12, s));
        // an asynchronous evaluation keeps the flags of earlier ones: they stay
        // set until airebo_check reads and clears them
        if (!async) CK(cudaMemsetAsync(h->derr, 0, sizeof(int) * 8, s));
        StepArgs<R> a = make_args<R>(h, pr, d_pos, d_force, d_w6 != nullptr);
        if (a.fix && h->n) CK(cudaMemsetAsync(a.fix, 0, sizeof(unsigned long long) * 3 * h->n, s));
        a.pgrad = d_pgrad;
        if (d_pgrad) CK(cudaMemsetAsync(d_pgrad, 0, sizeof(double) * 6, s));
        a.jv = d_jv;
        a.jout = d_jv ? d_jout : nullptr;
        if (d_jv) CK(cudaMemsetAsync(d_jout, 0, sizeof(double) * 6, s));
        if (d_kg) {
            // a second device copy of the parameters that carries the gradient buffer
            if (!pr.b.Pkg) CK(realloc_dev(pr.b.Pkg, 1));
            DevParams<R> pk = pr.hp;
            pk.kg = d_kg;
            CK(cudaStreamSynchronize(s));
            CK(cudaMemcpy(pr.b.Pkg, &pk, sizeof(DevParams<R>), cudaMemcpyHostToDevice));
            CK(cudaMemsetAsync(d_kg, 0, sizeof(double) * KG_N, s));
            a.P = pr.b.Pkg;
        }
        if (d_esys || d_eatom) {
            a.eatom = d_eatom ? d_eatom : h->eatom;
            if (h->n) CK(cudaMemsetAsync(a.eatom, 0, sizeof(double) * h->n, s));
        }
        launch_compute<R>(a, s, h->num_sms, (h->timing && !async) ? h->ev : nullptr);
        CK(cudaGetLastError());
        if (d_e4 || d_w6) k_finalize<<<1, 32, 0, s>>>(h->acc, d_e4, d_w6);
        if (d_esys) launch_system_energy(a.eatom, h->d_off, std::max(h->nsys, 1), d_esys, s);
        if (async) return AIREBO_OK;
        CK(cudaMemcpyAsync(h->h_err, h->derr, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h->h_u64, h->counts, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->timing && h->n) {
            // slot k: events k -> k+1; the second b* kernel (events 6 -> 7) is slot 8
            bool ran[7] = {true, a.rebo, a.torsion, a.lj_on, a.lj_on, a.lj_on, a.lj_on};
            for (int k = 0; k < 7; k++) {
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
                int slot = k == 6 ? 8 : k;
                if (ran[k]) { h->kt_ms[slot] += ms; h->kt_n[slot] += 1; }
            }
        }
        if (airebo_status st = device_errors(h)) return st;
        bool again = false;
        if (h->h_err[ERR_SHORT] > h->stride) {
            if (h->h_err[ERR_SHORT] > MAXN)
                return fail(h, AIREBO_ERR_CAPACITY, "an atom has more than " + std::to_string(MAXN) +
                                                    " REBO neighbours (" + std::to_string(h->h_err[ERR_SHORT]) + ")");
            h->stride = MAXN;
            airebo_status st = alloc_step<R>(h, pr, h->n_alloc);
            if (st) return st;
            again = true;
        }
        if (h->h_err[ERR_MAP]) {
            airebo_status st = grow_map<R>(h, pr, h->h_err[ERR_MAP]);
            if (st) return st;
            again = true;
        }
        const int* cn = (const int*)h->h_u64;
        int nq = std::max(std::max(cn[3], cn[4]), std::max(cn[5], cn[6]));    // path queue, b* queues
        if (nq > h->bq_cap) {
            h->bq_cap = nq + nq / 4 + 1024;
            CK(realloc_dev(h->bq, 3 * (size_t)h->bq_cap));
            CK(realloc_dev(h->bq2, 3 * (size_t)h->bq_cap));
            CK(realloc_dev(h->pq, (size_t)h->bq_cap));
            again = true;
        }
        if (!again) return AIREBO_OK;
    }
    return fail(h, AIREBO_ERR_CAPACITY, "scratch capacity did not converge");
}

airebo_status compute_any(airebo_handle h, const double* d_pos, double* d_force, double* d_e4, double* d_w6,
                          double* d_pgrad = nullptr, double* d_esys = nullptr, bool async = false,
                          double* d_kg = nullptr, double* d_eatom = nullptr, const double* d_jv = nullptr,
                          double* d_jout = nullptr) {
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_compute before airebo_neighbor");
    CK(cudaSetDevice(h->device));
    if (d_esys && !d_eatom && (h->eatom_n < h->n || !h->eatom)) {
        if (async) return fail(h, AIREBO_ERR_STATE, "per-system energies need one synchronous evaluation first");
        CK(realloc_dev(h->eatom, std::max(h->n, 1)));
        h->eatom_n = h->n;
    }
    if (h->opt.precision == AIREBO_MIXED)
        return do_compute<float>(h, h->p32, d_pos, d_force, d_e4, d_w6, d_pgrad, d_esys, async, d_kg, d_eatom, d_jv,
                                 d_jout);
    return do_compute<double>(h, h->p64, d_pos, d_force, d_e4, d_w6, d_pgrad, d_esys, async, d_kg, d_eatom, d_jv,
                              d_jout);
}

airebo_status check_rebuild(airebo_handle h, const double* d_pos, int* flag) {
    CK(cudaMemsetAsync(h->maxd2, 0, sizeof(unsigned long long), h->stream));
    launch_max_disp(d_pos, h->xref, h->n, h->maxd2, h->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_u64, h->maxd2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double d2;
    memcpy(&d2, h->h_u64, sizeof(double));
    double half = 0.5 * h->opt.skin;
    *flag = d2 > half * half ? 1 : 0;
    return AIREBO_OK;
}

// the split (hi on the 2^-12 A grid, lo the rest) of every system's box edges,
// for the image shifts of the LJ kernel on split positions
airebo_status upload_Lhl(airebo_handle h, const double* boxes, int nsys) {
    std::vector<float4> v(2 * (size_t)nsys);
    for (int s = 0; s < nsys; s++) {
        float hi[3], lo[3];
        for (int d = 0; d < 3; d++) {
            double q = std::rint(boxes[3 * s + d] * 4096.0) / 4096.0;
            hi[d] = (float)q;
            lo[d] = (float)(boxes[3 * s + d] - q);
        }
        v[2 * s] = make_float4(hi[0], hi[1], hi[2], 0.0f);
        v[2 * s + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
    }
    CK(realloc_dev(h->d_Lhl, v.size()));
    CK(cudaMemcpy(h->d_Lhl, v.data(), sizeof(float4) * v.size(), cudaMemcpyHostToDevice));
    return AIREBO_OK;
}

airebo_status set_system(airebo_handle h, const int8_t* d_types, int64_t n, const double* box, bool types_on_host) {
    if (n < 0 || n >= MAP_MAX_ATOMS) return fail(h, AIREBO_ERR_ARG, "atom count out of range (at most 2^28 - 1)");
    if (!box) return fail(h, AIREBO_ERR_ARG, "box is null");
    double dm = max3(h->sc.Dmax);
    for (int d = 0; d < 3; d++)
        if (!(box[d] > 4.0 * dm)) return fail(h, AIREBO_ERR_ARG, "box edge must exceed 4 x the largest REBO cut-off");
    airebo_status st = alloc_atoms(h, (int)n);
    if (st) return st;
    h->n = (int)n;
    h->nsys = 0;
    h->off_h.assign({0, (long long)n});
    CK(realloc_dev(h->d_off, 2));
    CK(cudaMemcpy(h->d_off, h->off_h.data(), sizeof(long long) * 2, cudaMemcpyHostToDevice));
    for (int d = 0; d < 3; d++) h->L[d] = box[d];
    st = upload_Lhl(h, box, 1);
    if (st) return st;
    if (n) CK(cudaMemcpyAsync(h->types, d_types, n, types_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
    return AIREBO_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

void airebo_default_options(airebo_options* o) {
    if (!o) return;
    o->skin = 1.0;
    o->precision = AIREBO_FP64;
    o->enable_rebo = 1;
    o->enable_lj = 1;
    o->enable_torsion = 1;
    o->max_lj_nbrs = 0;
    o->bstar_screen = 1;
}

airebo_status airebo_create(const char* params, const airebo_options* opts, void* stream, airebo_handle* out) {
    if (!params || !out) return AIREBO_ERR_ARG;
    *out = nullptr;
    airebo_handle h = new airebo_ctx();
    if (opts) h->opt = *opts; else airebo_default_options(&h->opt);
    if (!(h->opt.skin >= 0.0) ||
        (h->opt.precision != AIREBO_FP64 && h->opt.precision != AIREBO_MIXED && h->opt.precision != AIREBO_DF64)) {
        delete h;
        return AIREBO_ERR_ARG;
    }
    h->stream = (cudaStream_t)stream;
    HostParams hp;
    std::string e;
    if (!parse_text(params, hp, e) || !load_scalars(hp, h->sc, e)) {
        delete h;
        return AIREBO_ERR_ARG;
    }
    airebo_status st = AIREBO_OK;
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (ce != cudaSuccess) { delete h; return AIREBO_ERR_CUDA; }
    st = upload_own_params(h);
    if (!st) {
        if (realloc_dev(h->counts, 12) || realloc_dev(h->acc, 9) || realloc_dev(h->counters, 8) ||
            realloc_dev(h->derr, 8) || realloc_dev(h->maxd2, 1) || realloc_dev(h->ke, 1) ||
            realloc_dev(h->gate, 1) || realloc_dev(h->d_builds, 1) || realloc_dev(h->nerr, 4) ||
            cudaMemset(h->derr, 0, sizeof(int) * 8) || cudaMemset(h->d_builds, 0, sizeof(long long)) ||
            cudaMemset(h->nerr, 0, sizeof(int) * 4) ||
            cudaMallocHost((void**)&h->h_err, sizeof(int) * 8) || cudaMallocHost((void**)&h->h_u64, sizeof(unsigned long long) * 8) ||
            cudaMallocHost((void**)&h->h_acc, sizeof(double) * 16))
            st = AIREBO_ERR_CUDA;
    }
    if (st) { airebo_destroy(h); return st; }
    *out = h;
    return AIREBO_OK;
}

void airebo_destroy(airebo_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    free_prec(h->p64);
    free_prec(h->p32);
    free_prec(h->pdd);
    free_prec(h->pef);
    if (h->pg) cudaFree(h->pg);
    if (h->kg) cudaFree(h->kg);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    {
        void* bs[] = {h->d_sys, h->d_snc, h->d_sreach, h->d_scell0, h->d_Lsys, h->d_scw, h->d_off, h->eatom, h->d_Lhl};
        for (void* p : bs) if (p) cudaFree(p);
    }
    void* ps[] = {h->types, h->cell_of, h->cell_count, h->cell_start, h->cell_fill, h->spos, h->posf, h->pq_lo, h->fix, h->swrap, h->lj, h->lj_cnt,
                  h->im, h->im_cnt, h->xref, h->bonds, h->ccbonds, h->bq, h->bq2, h->pq, h->counts, h->acc, h->counters, h->derr, h->maxd2, h->ke,
                  h->gate, h->d_builds, h->nerr,
                  h->hpos, h->hvel, h->hforce, h->he4, h->hw6};
    for (void* p : ps) if (p) cudaFree(p);
    for (int k = 0; k < 12; k++) if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    if (h->h_err) cudaFreeHost(h->h_err);
    if (h->h_u64) cudaFreeHost(h->h_u64);
    if (h->h_acc) cudaFreeHost(h->h_acc);
    delete h;
}

const char* airebo_last_error(airebo_handle h) { return h ? h->err.c_str() : "null handle"; }

airebo_status airebo_neighbor(airebo_handle h, const double* d_pos, const int8_t* d_types, int64_t n, const double* box) {
    if (!h) return AIREBO_ERR_ARG;
    if (n > 0 && (!d_pos || !d_types)) return fail(h, AIREBO_ERR_ARG, "null position or type pointer");
    CK(cudaSetDevice(h->device));
    airebo_status st = set_system(h, d_types, n, box, false);
    if (st) return st;
    return do_neighbor(h, d_pos);
}

airebo_status airebo_compute(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4, double* d_virial6,
                             double* d_energy_per_atom) {
    if (!h) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    return compute_any(h, d_pos, d_force, d_energy4, d_virial6, nullptr, nullptr, false, nullptr, d_energy_per_atom);
}

airebo_status airebo_needs_rebuild(airebo_handle h, const double* d_pos, int* out_flag) {
    if (!h || !out_flag) return AIREBO_ERR_ARG;
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "no neighbour list yet");
    CK(cudaSetDevice(h->device));
    return check_rebuild(h, d_pos, out_flag);
}

static airebo_status stage_host(airebo_handle h, int n) {
    if (h->host_n == n && h->hpos) return AIREBO_OK;
    size_t m = 3 * (size_t)std::max(n, 1);
    CK(realloc_dev(h->hpos, m)); CK(realloc_dev(h->hvel, m)); CK(realloc_dev(h->hforce, m));
    CK(realloc_dev(h->he4, 4)); CK(realloc_dev(h->hw6, 6));
    h->host_n = n;
    return AIREBO_OK;
}

airebo_status airebo_compute_host(airebo_handle h, const double* h_pos, const int8_t* h_types, int64_t n,
                                  const double* box, double* h_force, double* h_energy4, double* h_virial6,
                                  double* h_energy_per_atom) {
    if (!h) return AIREBO_ERR_ARG;
    if (n > 0 && (!h_pos || !h_types || !h_force)) return fail(h, AIREBO_ERR_ARG, "null host pointer");
    CK(cudaSetDevice(h->device));
    airebo_status st = stage_host(h, (int)n);
    if (st) return st;
    if (n) CK(cudaMemcpyAsync(h->hpos, h_pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    bool rebuild = !h->built || n != h->n || !box || box[0] != h->L[0] || box[1] != h->L[1] || box[2] != h->L[2];
    if (rebuild) {
        st = set_system(h, h_types, n, box, true);
        if (st) return st;
        st = do_neighbor(h, h->hpos);
        if (st) return st;
    } else {
        int flag = 0;
        st = check_rebuild(h, h->hpos, &flag);
        if (st) return st;
        if (flag) { st = do_neighbor(h, h->hpos); if (st) return st; }
    }
    if (h_energy_per_atom && (h->eatom_n < h->n || !h->eatom)) {
        CK(realloc_dev(h->eatom, std::max(h->n, 1)));
        h->eatom_n = h->n;
    }
    st = compute_any(h, h->hpos, h->hforce, h->he4, h_virial6 ? h->hw6 : nullptr, nullptr, nullptr, false, nullptr,
                     h_energy_per_atom ? h->eatom : nullptr);
    if (st) return st;
    if (n) CK(cudaMemcpyAsync(h_force, h->hforce, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream));
    if (n && h_energy_per_atom)
        CK(cudaMemcpyAsync(h_energy_per_atom, h->eatom, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    if (h_energy4) CK(cudaMemcpyAsync(h_energy4, h->he4, sizeof(double) * 4, cudaMemcpyDeviceToHost, h->stream));
    if (h_virial6) CK(cudaMemcpyAsync(h_virial6, h->hw6, sizeof(double) * 6, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return AIREBO_OK;
}

// potential, kinetic and total energy, and the list builds so far: those the
// host ran plus those the device decided in asynchronous steps
__global__ void k_nve_energy(const double* acc, const double* ke, double* e4, long long rebuilds,
                             const long long* dev_builds) {
    if (threadIdx.x == 0) {
        double pe = acc[0] + acc[1] + acc[2];
        e4[0] = pe; e4[1] = *ke; e4[2] = pe + *ke; e4[3] = (double)(rebuilds + *dev_builds);
    }
}

airebo_status airebo_nve(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt, int nsteps,
                         double* d_energy4) {
    if (!h) return AIREBO_ERR_ARG;
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_nve before airebo_neighbor");
    if (nsteps < 0 || !(dt > 0)) return fail(h, AIREBO_ERR_ARG, "bad dt or step count");
    CK(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    bool pending = false;      // second half step timed but not yet read
    auto read_pending = [&]() -> airebo_status {
        if (pending) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, h->ev[10], h->ev[11]));
            h->kt_ms[7] += ms;
            h->kt_n[7] += 1;
            pending = false;
        }
        return AIREBO_OK;
    };
    for (int step = 0; step < nsteps; step++) {
        CK(cudaMemsetAsync(h->maxd2, 0, sizeof(unsigned long long), s));
        if (h->timing) CK(cudaEventRecord(h->ev[8], s));
        launch_nve_half(d_pos, d_vel, d_force, h->types, h->n, dt, true, h->xref, h->maxd2, nullptr, s);
        CK(cudaGetLastError());
        if (h->timing) CK(cudaEventRecord(h->ev[9], s));
        CK(cudaMemcpyAsync(h->h_u64, h->maxd2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->timing) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, h->ev[8], h->ev[9]));
            h->kt_ms[7] += ms;
            h->kt_n[7] += 1;
            airebo_status st = read_pending();
            if (st) return st;
        }
        double d2;
        memcpy(&d2, h->h_u64, sizeof(double));
        double half = 0.5 * h->opt.skin;
        if (d2 > half * half) {
            airebo_status st = do_neighbor(h, d_pos);
            if (st) return st;
        }
        bool last = step == nsteps - 1;
        airebo_status st = compute_any(h, d_pos, d_force, nullptr, nullptr);
        if (st) return st;
        if (last) CK(cudaMemsetAsync(h->ke, 0, sizeof(double), s));
        if (h->timing) CK(cudaEventRecord(h->ev[10], s));
        launch_nve_half(d_pos, d_vel, d_force, h->types, h->n, dt, false, nullptr, nullptr, last ? h->ke : nullptr, s);
        CK(cudaGetLastError());
        if (h->timing) { CK(cudaEventRecord(h->ev[11], s)); pending = true; }
        if (last && d_energy4) k_nve_energy<<<1, 32, 0, s>>>(h->acc, h->ke, d_energy4, h->rebuilds, h->d_builds);
    }
    CK(cudaGetLastError());
    if (pending) {
        CK(cudaEventSynchronize(h->ev[11]));
        airebo_status st = read_pending();
        if (st) return st;
    }
    return AIREBO_OK;
}

airebo_status airebo_nve_host(airebo_handle h, double* h_pos, double* h_vel, double* h_force, double dt, int nsteps,
                              double* h_energy4) {
    if (!h) return AIREBO_ERR_ARG;
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_nve_host before a neighbour build");
    int n = h->n;
    if (n > 0 && (!h_pos || !h_vel || !h_force)) return fail(h, AIREBO_ERR_ARG, "null host pointer");
    CK(cudaSetDevice(h->device));
    airebo_status st = stage_host(h, n);
    if (st) return st;
    size_t bytes = sizeof(double) * 3 * n;
    cudaStream_t s = h->stream;
    if (n) {
        CK(cudaMemcpyAsync(h->hpos, h_pos, bytes, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->hvel, h_vel, bytes, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->hforce, h_force, bytes, cudaMemcpyHostToDevice, s));
    }
    st = airebo_nve(h, h->hpos, h->hvel, h->hforce, dt, nsteps, h->he4);
    if (st) return st;
    if (n) {
        CK(cudaMemcpyAsync(h_pos, h->hpos, bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_vel, h->hvel, bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_force, h->hforce, bytes, cudaMemcpyDeviceToHost, s));
    }
    if (h_energy4) CK(cudaMemcpyAsync(h_energy4, h->he4, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return AIREBO_OK;
}

airebo_status airebo_counters(airebo_handle h, int64_t* out8) {
    if (!h || !out8) return AIREBO_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(h->h_u64, h->counters, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, h->stream));
    long long dev_builds = 0;
    CK(cudaMemcpyAsync(&dev_builds, h->d_builds, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 8; k++) out8[k] = (int64_t)h->h_u64[k];
    out8[5] = h->rebuilds + dev_builds;
    out8[6] = h->lj_cap;
    int mc = h->opt.precision == AIREBO_MIXED ? h->p32.b.map_cap : h->p64.b.map_cap;
    out8[4] = mc;
    return AIREBO_OK;
}

airebo_status airebo_neighbor_batch(airebo_handle h, const double* d_pos, const int8_t* d_types, int64_t n,
                                    int nsys, const int64_t* h_offsets, const double* h_boxes) {
    if (!h || nsys < 1 || !h_offsets || !h_boxes) return AIREBO_ERR_ARG;
    if (n > 0 && (!d_pos || !d_types)) return fail(h, AIREBO_ERR_ARG, "null position or type pointer");
    if (h_offsets[0] != 0 || h_offsets[nsys] != n) return fail(h, AIREBO_ERR_ARG, "offsets must run from 0 to n");
    double dm = max3(h->sc.Dmax);
    for (int s = 0; s < nsys; s++) {
        if (h_offsets[s + 1] < h_offsets[s]) return fail(h, AIREBO_ERR_ARG, "offsets must not decrease");
        for (int d = 0; d < 3; d++)
            if (!(h_boxes[3 * s + d] > 4.0 * dm))
                return fail(h, AIREBO_ERR_ARG, "box edge must exceed 4 x the largest REBO cut-off");
    }
    CK(cudaSetDevice(h->device));
    airebo_status st = set_system(h, d_types, n, h_boxes, false);
    if (st) return st;
    h->nsys = nsys;
    h->Lsys_h.assign(h_boxes, h_boxes + 3 * nsys);
    h->off_h.assign(h_offsets, h_offsets + nsys + 1);
    std::vector<int> sys((size_t)std::max<int64_t>(n, 1));
    for (int s = 0; s < nsys; s++)
        for (int64_t i = h_offsets[s]; i < h_offsets[s + 1]; i++) sys[i] = s;
    CK(realloc_dev(h->d_sys, sys.size()));
    CK(realloc_dev(h->d_Lsys, 3 * (size_t)nsys));
    CK(realloc_dev(h->d_snc, 3 * (size_t)nsys));
    CK(realloc_dev(h->d_sreach, 3 * (size_t)nsys));
    CK(realloc_dev(h->d_scw, 3 * (size_t)nsys));
    CK(realloc_dev(h->d_scell0, (size_t)nsys + 1));
    CK(realloc_dev(h->d_off, (size_t)nsys + 1));
    CK(cudaMemcpy(h->d_sys, sys.data(), sizeof(int) * sys.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_Lsys, h_boxes, sizeof(double) * 3 * nsys, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_off, h->off_h.data(), sizeof(long long) * (nsys + 1), cudaMemcpyHostToDevice));
    st = upload_Lhl(h, h_boxes, nsys);
    if (st) return st;
    return do_neighbor(h, d_pos);
}

airebo_status airebo_compute_batch(airebo_handle h, const double* d_pos, double* d_force, double* d_energy_sys) {
    if (!h || !d_energy_sys) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    return compute_any(h, d_pos, d_force, nullptr, nullptr, nullptr, d_energy_sys, false);
}

airebo_status airebo_compute_async(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                                   double* d_energy_sys) {
    if (!h) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    return compute_any(h, d_pos, d_force, d_energy4, nullptr, nullptr, d_energy_sys, true);
}

airebo_status airebo_check(airebo_handle h) {
    if (!h) return AIREBO_ERR_ARG;
    CK(cudaSetDevice(h->device));
    CK(cudaMemcpyAsync(h->h_err, h->derr, sizeof(int) * 8, cudaMemcpyDeviceToHost, h->stream));
    int nerr[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(nerr, h->nerr, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // read once: the flags of the asynchronous work so far start again from zero
    CK(cudaMemsetAsync(h->derr, 0, sizeof(int) * 8, h->stream));
    CK(cudaMemsetAsync(h->nerr, 0, sizeof(int) * 4, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // the list builds the device decided on in asynchronous MD steps
    if (nerr[2] == 1) return fail(h, AIREBO_ERR_NONFINITE, "non-finite position at a list build");
    if (nerr[2] == 2) return fail(h, AIREBO_ERR_ARG, "position more than 120 box lengths outside the box at a list build");
    if (nerr[3]) return fail(h, AIREBO_ERR_ARG, "atom type other than 0 (C) or 1 (H)");
    if (airebo_status st = device_errors(h)) return st;
    if (nerr[0] > h->lj_cap || nerr[1] > h->im_cap)
        return fail(h, AIREBO_ERR_CAPACITY, "a neighbour-list capacity was exceeded at a list build; run airebo_neighbor and "
                                            "airebo_compute once to grow it");
    std::string cap;
    if (h->h_err[ERR_SHORT] > h->stride) cap += " REBO neighbours per atom (" + std::to_string(h->h_err[ERR_SHORT]) + ")";
    if (h->h_err[ERR_MAP]) cap += " connectivity-map entries per atom (" + std::to_string(h->h_err[ERR_MAP]) + ")";
    if (h->h_err[ERR_QUEUE] > h->bq_cap) cap += " b* or path queue (" + std::to_string(h->h_err[ERR_QUEUE]) + ")";
    if (!cap.empty())
        return fail(h, AIREBO_ERR_CAPACITY, "a scratch capacity was exceeded:" + cap + "; run airebo_compute once to grow it");
    return AIREBO_OK;
}

}  // extern "C"

// Headroom for work that cannot grow a capacity while it runs (captured MD
// steps): the full REBO slot stride, a quarter more connectivity-map entries
// per atom, and a quarter more b* queue than the last evaluation needed.
template <class R> static airebo_status reserve_headroom(airebo_handle h, Precision<R>& pr) {
    if (h->stride < MAXN) {
        h->stride = MAXN;
        airebo_status st = alloc_step<R>(h, pr, h->n_alloc);
        if (st) return st;
    }
    StepBuffers<R>& b = pr.b;
    b.map_cap += b.map_cap / 4 + 4;
    if (airebo_status st2 = alloc_map<R>(h, b, h->n_alloc)) return st2;
    CK(cudaMemcpyAsync(h->h_u64, h->counts, sizeof(int) * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int* cn = (const int*)h->h_u64;
    int nq = std::max(std::max(cn[3], cn[4]), std::max(cn[5], cn[6]));
    if (nq + nq / 4 + 1024 > h->bq_cap) {
        h->bq_cap = nq + nq / 4 + 1024;
        CK(realloc_dev(h->bq, 3 * (size_t)h->bq_cap));
        CK(realloc_dev(h->bq2, 3 * (size_t)h->bq_cap));
        CK(realloc_dev(h->pq, (size_t)h->bq_cap));
    }
    return AIREBO_OK;
}

extern "C" {

// One velocity-Verlet step with no host work: the half kick and drift with the
// displacement check, the device's rebuild decision, the list build behind it,
// the evaluation, and the second half kick.
static airebo_status nve_step_async(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt,
                                    bool last, double* d_energy4) {
    cudaStream_t s = h->stream;
    CK(cudaMemsetAsync(h->maxd2, 0, sizeof(unsigned long long), s));
    launch_nve_half(d_pos, d_vel, d_force, h->types, h->n, dt, true, h->xref, h->maxd2, nullptr, s);
    double half = 0.5 * h->opt.skin;
    launch_rebuild_decide(h->maxd2, half * half, h->gate, h->d_builds, s);
    NeighborArgs a = h->nargs;
    a.pos = d_pos;
    a.err = h->nerr;
    a.gate = h->gate;
    launch_neighbor_gated(a, s, h->nargs_ncell);
    CK(cudaGetLastError());
    airebo_status st = compute_any(h, d_pos, d_force, nullptr, nullptr, nullptr, nullptr, true);
    if (st) return st;
    if (last) CK(cudaMemsetAsync(h->ke, 0, sizeof(double), s));
    launch_nve_half(d_pos, d_vel, d_force, h->types, h->n, dt, false, nullptr, nullptr, last ? h->ke : nullptr, s);
    if (last && d_energy4) k_nve_energy<<<1, 32, 0, s>>>(h->acc, h->ke, d_energy4, h->rebuilds, h->d_builds);
    CK(cudaGetLastError());
    return AIREBO_OK;
}

airebo_status airebo_nve_async(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt, int nsteps,
                               double* d_energy4) {
    if (!h) return AIREBO_ERR_ARG;
    if (!h->built || !h->nargs_ok) return fail(h, AIREBO_ERR_STATE, "airebo_nve_async before airebo_neighbor");
    if (nsteps < 0 || !(dt > 0)) return fail(h, AIREBO_ERR_ARG, "bad dt or step count");
    if (h->n > 0 && (!d_pos || !d_vel || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position, velocity or force pointer");
    CK(cudaSetDevice(h->device));
    for (int step = 0; step < nsteps; step++) {
        airebo_status st = nve_step_async(h, d_pos, d_vel, d_force, dt, step == nsteps - 1, d_energy4);
        if (st) return st;
    }
    return AIREBO_OK;
}

airebo_status airebo_graph_capture_nve(airebo_handle h, double* d_pos, double* d_vel, double* d_force, double dt,
                                       int nsteps, double* d_energy4) {
    if (!h) return AIREBO_ERR_ARG;
    if (!h->stream) return fail(h, AIREBO_ERR_ARG, "graph capture needs a handle created on a non-default stream");
    if (!h->built || !h->nargs_ok) return fail(h, AIREBO_ERR_STATE, "airebo_graph_capture_nve before airebo_neighbor");
    if (nsteps < 1 || !(dt > 0)) return fail(h, AIREBO_ERR_ARG, "bad dt or step count");
    if (h->n > 0 && (!d_pos || !d_vel || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position, velocity or force pointer");
    CK(cudaSetDevice(h->device));
    // the lists are rebuilt at d_pos with a quarter more room per atom, a
    // synchronous evaluation grows every scratch capacity, the scratch gets
    // headroom for the steps ahead too, and a second evaluation leaves in
    // d_force the forces the first step starts from
    if (h->opt.enable_lj) h->lj_cap = ((int)(h->lj_cap * 1.25) + 31) / 32 * 32;
    h->im_cap += h->im_cap / 4 + 4;
    airebo_status st = do_neighbor(h, d_pos);
    if (st) return st;
    st = compute_any(h, d_pos, d_force, nullptr, nullptr);
    if (st) return st;
    st = h->opt.precision == AIREBO_MIXED ? reserve_headroom<float>(h, h->p32) : reserve_headroom<double>(h, h->p64);
    if (st) return st;
    st = compute_any(h, d_pos, d_force, nullptr, nullptr);
    if (st) return st;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    st = airebo_nve_async(h, d_pos, d_vel, d_force, dt, nsteps, d_energy4);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return fail(h, AIREBO_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    h->graph = g;
    CK(cudaGraphInstantiate(&h->gexec, g, 0));
    return AIREBO_OK;
}

airebo_status airebo_graph_capture(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                                   double* d_energy_sys) {
    if (!h) return AIREBO_ERR_ARG;
    if (!h->stream) return fail(h, AIREBO_ERR_ARG, "graph capture needs a handle created on a non-default stream");
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_graph_capture before airebo_neighbor");
    CK(cudaSetDevice(h->device));
    // one synchronous evaluation grows every capacity the graph will need
    airebo_status st = compute_any(h, d_pos, d_force, d_energy4, nullptr, nullptr, d_energy_sys, false);
    if (st) return st;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    st = compute_any(h, d_pos, d_force, d_energy4, nullptr, nullptr, d_energy_sys, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return fail(h, AIREBO_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    h->graph = g;
    CK(cudaGraphInstantiate(&h->gexec, g, 0));
    return AIREBO_OK;
}

airebo_status airebo_graph_launch(airebo_handle h) {
    if (!h) return AIREBO_ERR_ARG;
    if (!h->gexec) return fail(h, AIREBO_ERR_STATE, "no captured graph");
    CK(cudaSetDevice(h->device));
    CK(cudaGraphLaunch(h->gexec, h->stream));
    return AIREBO_OK;
}

airebo_status airebo_autotune(airebo_handle h, const double* d_pos, double* d_force, int* out3) {
    if (!h) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_autotune before airebo_neighbor");
    CK(cudaSetDevice(h->device));
    bool was_timing = h->timing;
    airebo_status st = airebo_set_timing(h, 1);
    if (st) return st;
    st = compute_any(h, d_pos, d_force, nullptr, nullptr);        // settle every capacity first
    if (st) return st;
    // median over REPS evaluations of the kernel times k0..k1 (event indices)
    const int REPS = 5;
    auto timed = [&](double* med_a, double* med_b) -> airebo_status {
        double ta[REPS], tb[REPS];
        for (int rep = 0; rep < REPS; rep++) {
            for (int k = 0; k < 9; k++) { h->kt_ms[k] = 0; h->kt_n[k] = 0; }
            airebo_status s2 = compute_any(h, d_pos, d_force, nullptr, nullptr);
            if (s2) return s2;
            ta[rep] = h->kt_ms[4];                       // LJ
            tb[rep] = h->kt_ms[1] + h->kt_ms[2];         // REBO + torsion
            if (med_b) med_b[rep] = h->kt_ms[5] + h->kt_ms[8];   // both b* kernels
        }
        std::sort(ta, ta + REPS);
        std::sort(tb, tb + REPS);
        med_a[0] = ta[REPS / 2];
        med_a[1] = tb[REPS / 2];
        if (med_b) std::sort(med_b, med_b + REPS);
        return AIREBO_OK;
    };
    const int chunks[] = {2, 4, 8, 16};
    const int waves[] = {2, 4, 8, 16, 32};
    double best_lj = 1e300, best_bond = 1e300, best_bstar = 1e300;
    int bc = h->lj_chunk, bg = h->bond_waves, bs = h->bstar_waves;
    // the LJ chunk and the two grids act on different kernels: tune each
    if (h->opt.enable_lj) {
        for (int c : chunks) {
            h->lj_chunk = c;
            double m[2];
            st = timed(m, nullptr);
            if (st) return st;
            if (m[0] < best_lj) { best_lj = m[0]; bc = c; }
        }
    }
    h->lj_chunk = bc;
    for (int g : waves) {
        h->bond_waves = g;
        h->bstar_waves = g;
        double m[2], tb[REPS];
        st = timed(m, tb);
        if (st) return st;
        if (m[1] < best_bond) { best_bond = m[1]; bg = g; }
        if (tb[REPS / 2] < best_bstar) { best_bstar = tb[REPS / 2]; bs = g; }
    }
    h->bond_waves = bg;
    h->bstar_waves = bs;
    airebo_set_timing(h, was_timing ? 1 : 0);
    if (out3) { out3[0] = h->lj_chunk; out3[1] = h->bond_waves; out3[2] = h->bstar_waves; }
    return AIREBO_OK;
}

airebo_status airebo_set_launch_shape(airebo_handle h, int lj_chunk, int bond_waves, int bstar_waves) {
    if (!h) return AIREBO_ERR_ARG;
    if (lj_chunk < 1 || lj_chunk > 64 || bond_waves < 1 || bond_waves > 32 || bstar_waves < 1 || bstar_waves > 32)
        return fail(h, AIREBO_ERR_ARG, "launch shape out of range (lj_chunk 1..64, waves 1..32)");
    h->lj_chunk = lj_chunk;
    h->bond_waves = bond_waves;
    h->bstar_waves = bstar_waves;
    return AIREBO_OK;
}

airebo_status airebo_param_grad(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                                double* h_grad6) {
    if (!h || !h_grad6) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_param_grad before airebo_neighbor");
    CK(cudaSetDevice(h->device));
    if (!h->pg) CK(realloc_dev(h->pg, 12));
    airebo_status st = compute_any(h, d_pos, d_force, d_energy4, nullptr, h->pg);
    if (st) return st;
    CK(cudaMemcpyAsync(h->h_acc, h->pg, sizeof(double) * 6, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 6; k++) h_grad6[k] = h->h_acc[k];
    return AIREBO_OK;
}

airebo_status airebo_force_param_grad(airebo_handle h, const double* d_pos, const double* d_v, double* d_force,
                                      double* d_energy4, double* h_out6) {
    if (!h || !h_out6) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force || !d_v)) return fail(h, AIREBO_ERR_ARG, "null position, direction or force pointer");
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_force_param_grad before airebo_neighbor");
    CK(cudaSetDevice(h->device));
    if (!h->pg) CK(realloc_dev(h->pg, 12));
    airebo_status st = compute_any(h, d_pos, d_force, d_energy4, nullptr, nullptr, nullptr, false, nullptr, nullptr,
                                   d_v, h->pg + 6);
    if (st) return st;
    CK(cudaMemcpyAsync(h->h_acc, h->pg + 6, sizeof(double) * 6, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 6; k++) h_out6[k] = h->h_acc[k];
    return AIREBO_OK;
}

airebo_status airebo_knot_grad(airebo_handle h, const double* d_pos, double* d_force, double* d_energy4,
                               double* h_grad, int64_t count) {
    if (!h || !h_grad) return AIREBO_ERR_ARG;
    if (count != AIREBO_KNOT_COUNT) return fail(h, AIREBO_ERR_ARG, "knot gradient needs AIREBO_KNOT_COUNT values");
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_knot_grad before airebo_neighbor");
    CK(cudaSetDevice(h->device));
    if (!h->kg) CK(realloc_dev(h->kg, KG_N));
    airebo_status st = compute_any(h, d_pos, d_force, d_energy4, nullptr, nullptr, nullptr, false, h->kg);
    if (st) return st;
    std::vector<double> g(KG_N, 0.0);
    CK(cudaMemcpyAsync(g.data(), h->kg, sizeof(double) * KG_N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // parameter-file order: gC1, gC2, gH, P.CC, P.CH, P.HC, piRC.CC, piRC.CH, piRC.HH, Tij.CC
    for (int64_t k = 0; k < count; k++) h_grad[k] = 0;
    const Scalars& sc = h->sc;
    double* o = h_grad;
    quintic_coeffs_adjoint(sc.gC1k, g.data() + KG_GC1, o); o += 3 * sc.gC1k.size();
    quintic_coeffs_adjoint(sc.gC2k, g.data() + KG_GC2, o); o += 3 * sc.gC2k.size();
    quintic_coeffs_adjoint(sc.gHk, g.data() + KG_GH, o); o += 3 * sc.gHk.size();
    for (int t = 0; t < 3; t++, o += 100) bicubic_coeffs_adjoint(g.data() + KG_P + t * 256, o);
    for (int t = 0; t < 3; t++, o += 1800) tricubic_coeffs_adjoint(g.data() + KG_F + t * NTRI_CELLS * 64, o);
    tricubic_coeffs_adjoint(g.data() + KG_T, o);
    return AIREBO_OK;
}

airebo_status airebo_set_lj_params(airebo_handle h, const double* eps3, const double* sigma3) {
    if (!h || (!eps3 && !sigma3)) return AIREBO_ERR_ARG;
    Scalars s = h->sc;
    bool sigma_changed = false;
    for (int p = 0; p < 3; p++) {
        if (eps3) {
            if (!(eps3[p] > 0)) return fail(h, AIREBO_ERR_ARG, "epsilon must be positive");
            if (s.kind == 0) s.eps[p] = eps3[p]; else s.meps[p] = eps3[p];
        }
        if (sigma3) {
            if (!(sigma3[p] > 0)) return fail(h, AIREBO_ERR_ARG, "sigma must be positive");
            sigma_changed |= sigma3[p] != s.sigma[p];
            s.sigma[p] = sigma3[p];
        }
    }
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    h->sc = s;
    airebo_status st = upload_own_params(h);
    if (st) return st;
    if (sigma_changed) h->built = false;          // the LJ cut-off moved: the lists must be rebuilt
    return AIREBO_OK;
}

airebo_status airebo_bstar_bound_check(airebo_handle h, const double* d_pos, double* d_force, double* h_out6) {
    if (!h || !h_out6) return AIREBO_ERR_ARG;
    if (h->n > 0 && (!d_pos || !d_force)) return fail(h, AIREBO_ERR_ARG, "null position or force pointer");
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "airebo_bstar_bound_check before airebo_neighbor");
    if (!screen_on(h)) return fail(h, AIREBO_ERR_STATE, "the b* screen is off on this handle");
    CK(cudaSetDevice(h->device));
    airebo_status st = compute_any(h, d_pos, d_force, nullptr, nullptr);
    if (st) return st;
    double* out = nullptr;
    CK(cudaMalloc((void**)&out, sizeof(double) * 6));
    CK(cudaMemsetAsync(out, 0, sizeof(double) * 6, h->stream));
    StepArgs<double> a = make_args<double>(h, h->p64, d_pos, d_force, false);
    if (h->n) launch_bstar_bound_check(a, out, h->stream, h->num_sms);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out6, out, sizeof(double) * 6, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(out);
    if (e != cudaSuccess) return fail(h, AIREBO_ERR_CUDA, cudaGetErrorString(e));
    return AIREBO_OK;
}

airebo_status airebo_set_knots(airebo_handle h, const double* h_knots, int64_t count) {
    if (!h || !h_knots) return AIREBO_ERR_ARG;
    if (count != AIREBO_KNOT_COUNT) return fail(h, AIREBO_ERR_ARG, "knot data need AIREBO_KNOT_COUNT values");
    for (int64_t k = 0; k < count; k++)
        if (!std::isfinite(h_knots[k])) return fail(h, AIREBO_ERR_ARG, "non-finite knot datum");
    Scalars s = h->sc;
    // the parameter-file order of airebo_knot_grad
    const double* q = h_knots;
    auto take = [&](std::vector<double>& dst) { std::copy(q, q + dst.size(), dst.begin()); q += dst.size(); };
    take(s.gC1d); take(s.gC2d); take(s.gHd);
    for (int t = 0; t < 3; t++) take(s.P[t]);
    for (int t = 0; t < 3; t++) take(s.F[t]);
    take(s.T);
    if (q - h_knots != count) return fail(h, AIREBO_ERR_ARG, "knot layout mismatch");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    Scalars old = h->sc;
    h->sc = s;
    airebo_status st = upload_own_params(h);
    if (st) { h->sc = old; upload_own_params(h); return st; }
    return AIREBO_OK;
}

airebo_status airebo_export_lists(airebo_handle h, int which, int32_t* h_cnt, int32_t* h_j, int8_t* h_img, int64_t cap) {
    if (!h || !h_cnt || !h_j || !h_img || cap < 0 || which < 0 || which > 2) return AIREBO_ERR_ARG;
    if (!h->built) return fail(h, AIREBO_ERR_STATE, "no neighbour list yet");
    CK(cudaSetDevice(h->device));
    CK(cudaStreamSynchronize(h->stream));
    int n = h->n;
    std::vector<int> cnt(n);
    std::vector<int2> ent;
    int rowcap = 0;
    if (which == 2) {
        const int* dcnt = h->opt.precision == AIREBO_MIXED ? h->p32.b.cnt : h->p64.b.cnt;
        const int* dnj = h->opt.precision == AIREBO_MIXED ? h->p32.b.nj : h->p64.b.nj;
        const int* dimg = h->opt.precision == AIREBO_MIXED ? h->p32.b.nimg : h->p64.b.nimg;
        rowcap = h->stride;
        std::vector<int> nj((size_t)n * h->stride), im((size_t)n * h->stride);
        if (n) {
            CK(cudaMemcpy(cnt.data(), dcnt, sizeof(int) * n, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(nj.data(), dnj, sizeof(int) * nj.size(), cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(im.data(), dimg, sizeof(int) * im.size(), cudaMemcpyDeviceToHost));
        }
        ent.resize(nj.size());
        for (size_t k = 0; k < nj.size(); k++) ent[k] = make_int2(nj[k], im[k]);
    } else {
        rowcap = which == 0 ? h->lj_cap : h->im_cap;
        ent.resize((size_t)n * rowcap);
        if (n) {
            CK(cudaMemcpy(cnt.data(), which == 0 ? h->lj_cnt : h->im_cnt, sizeof(int) * n, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(ent.data(), which == 0 ? h->lj : h->im, sizeof(int2) * ent.size(), cudaMemcpyDeviceToHost));
        }
    }
    for (int i = 0; i < n; i++) {
        h_cnt[i] = cnt[i];
        for (int e = 0; e < cnt[i] && e < cap; e++) {
            int2 v = ent[(size_t)i * rowcap + e];
            h_j[(size_t)i * cap + e] = v.x;
            h_img[((size_t)i * cap + e) * 3 + 0] = (int8_t)img_x(v.y);
            h_img[((size_t)i * cap + e) * 3 + 1] = (int8_t)img_y(v.y);
            h_img[((size_t)i * cap + e) * 3 + 2] = (int8_t)img_z(v.y);
        }
    }
    return AIREBO_OK;
}

airebo_status airebo_set_timing(airebo_handle h, int on) {
    if (!h) return AIREBO_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (on && !h->ev[0])
        for (int k = 0; k < 12; k++) CK(cudaEventCreate(&h->ev[k]));
    h->timing = on != 0;
    for (int k = 0; k < 9; k++) { h->kt_ms[k] = 0; h->kt_n[k] = 0; }
    return AIREBO_OK;
}

airebo_status airebo_kernel_times(airebo_handle h, double* ms, int64_t* launches) {
    if (!h || !ms || !launches) return AIREBO_ERR_ARG;
    for (int k = 0; k < 9; k++) { ms[k] = h->kt_ms[k]; launches[k] = h->kt_n[k]; }
    return AIREBO_OK;
}

airebo_status airebo_alu_peak(int precision, double* tflops) {
    if (!tflops || (precision != AIREBO_FP64 && precision != AIREBO_MIXED)) return AIREBO_ERR_ARG;
    double t = alu_peak(precision == AIREBO_FP64 ? 1 : 0);
    *tflops = t;
    return t > 0 ? AIREBO_OK : AIREBO_ERR_CUDA;
}

airebo_status airebo_math_check(int64_t* h_ulp4) {
    if (!h_ulp4) return AIREBO_ERR_ARG;
    long long o[4] = {0, 0, 0, 0};
    if (math_check(o)) return AIREBO_ERR_CUDA;
    for (int k = 0; k < 4; k++) h_ulp4[k] = o[k];
    return AIREBO_OK;
}

airebo_status airebo_dd_check(double* h_err8) {
    if (!h_err8) return AIREBO_ERR_ARG;
    if (dd_check(h_err8)) return AIREBO_ERR_CUDA;
    return AIREBO_OK;
}

}  // extern "C"
