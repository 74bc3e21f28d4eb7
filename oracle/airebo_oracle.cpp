// AIREBO CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow FP64 evaluation of the AIREBO energy (Sec. 2.1 of Hoehnerbach &
// Bientinesi, "Optimizing AIREBO"), used by the tests and by the CPU baseline of
// the bench to check the CUDA library.  It shares no code with the CUDA path.
// Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
// arm may load it; the library never does.
//
// What it computes (terms of Sec. 2.1; functional forms the paper does not
// print follow the readings listed in the design notes of the repository):
//   E = sum_{bonds i<j} [ f_R(r_ij) + b_ij f_A(r_ij) ]                    (REBO, Alg. 1)
//     + sum_{i<j bonds, C-C} sum_{k,l} w_ki w_ij w_jl V^tors(omega_kijl)   (torsion, Alg. 2)
//     + sum_{pairs i<j, images} (S_r S_b(b*_ij) + 1 - S_r) C_ij V^LJ(r_ij)  (LJ, Alg. 3)
//   b_ij = 1/2 (p_ij + p_ji) + pi^rc_ij + pi^dh_ij                        (Sec. 2.1.3)
//   p_ij = [1 + sum_k w_ik g_i(cos theta_jik) e^lambda_jik + P_ij]^(-1/2)   (Sec. 2.1.3)
//   C_ij = 1 - max{w_ij, w_ik w_kj, w_ik w_kl w_lj}                       (Sec. 2.1.2)
//
// Forces are the exact gradient of the energy as written here: every term is
// evaluated on a small reverse-mode tape (the forward/reverse pass pattern of
// Sec. 2), whose adjoints are the force contributions.  So the oracle needs no
// hand-derived derivative; finite differences of its energy pin the gradient.
//
// The C_ij search is the original nested loop over neighbours and their
// neighbours (Sec. 4.3), not a map; neighbour sets are found by plain binning
// with explicit periodic images (Sec. 2).
//
// Parity pins for every function here live in tests/test_oracle_*.py.

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <sstream>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// reverse-mode tape
// ---------------------------------------------------------------------------
struct Node { int a, b; double da, db; };
thread_local std::vector<Node> g_tape;

struct V {
    double v;
    int id;   // -1: constant
};
inline V cst(double x) { return V{x, -1}; }
inline V mk(double v, int a, double da, int b, double db) {
    if (a < 0 && b < 0) return cst(v);
    g_tape.push_back(Node{a, b, da, db});
    return V{v, (int)g_tape.size() - 1};
}
inline V leaf(double x) { g_tape.push_back(Node{-1, -1, 0.0, 0.0}); return V{x, (int)g_tape.size() - 1}; }
inline V operator+(V x, V y) { return mk(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline V operator-(V x, V y) { return mk(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline V operator*(V x, V y) { return mk(x.v * y.v, x.id, y.v, y.id, x.v); }
inline V operator/(V x, V y) { return mk(x.v / y.v, x.id, 1.0 / y.v, y.id, -x.v / (y.v * y.v)); }
inline V operator-(V x) { return mk(-x.v, x.id, -1.0, -1, 0.0); }
inline V operator+(V x, double y) { return mk(x.v + y, x.id, 1.0, -1, 0.0); }
inline V operator+(double y, V x) { return x + y; }
inline V operator-(V x, double y) { return mk(x.v - y, x.id, 1.0, -1, 0.0); }
inline V operator-(double y, V x) { return mk(y - x.v, x.id, -1.0, -1, 0.0); }
inline V operator*(V x, double y) { return mk(x.v * y, x.id, y, -1, 0.0); }
inline V operator*(double y, V x) { return x * y; }
inline V operator/(V x, double y) { return mk(x.v / y, x.id, 1.0 / y, -1, 0.0); }
inline V operator/(double y, V x) { return mk(y / x.v, x.id, -y / (x.v * x.v), -1, 0.0); }
inline V vexp(V x) { double e = std::exp(x.v); return mk(e, x.id, e, -1, 0.0); }
inline V vcos(V x) { return mk(std::cos(x.v), x.id, -std::sin(x.v), -1, 0.0); }
inline V vsqrt(V x) { double s = std::sqrt(x.v); return mk(s, x.id, 0.5 / s, -1, 0.0); }
inline V vpow(V x, double p) { return mk(std::pow(x.v, p), x.id, p * std::pow(x.v, p - 1.0), -1, 0.0); }

struct V3 { V x, y, z; };
inline V3 operator-(const V3& a, const V3& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(const V3& a, V s) { return {a.x * s, a.y * s, a.z * s}; }
inline V dot(const V3& a, const V3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(const V3& a, const V3& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline V norm(const V3& a) { return vsqrt(dot(a, a)); }

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
enum { CC = 0, CH = 1, HH = 2 };
inline int pair_index(int ti, int tj) { return ti + tj; }   // 0 CC, 1 CH/HC, 2 HH

struct Params {
    std::map<std::string, std::vector<double>> raw;
    double Dmin[3], Dmax[3], Q[3], alpha[3], A[3], B[3][3], beta[3][3], rho[3];
    double lam_coef, gN0, gN1, Fx0, Fx1;
    std::vector<double> gC1k, gC1d, gC2k, gC2d, gHk, gHd;
    std::vector<double> P[3];       // CC, CH, HC: 5x5x4
    std::vector<double> piRC[3];    // CC, CH, HH: 5x5x9x8
    std::vector<double> Tcc;        // 5x5x9x8
    double guard0, guard1;
    double sigma[3], eps[3], ljcut, ljsw, SrLo, SrHi;
    double bmin[3], bmax[3], rstar[3];
    double teps[3];
    int inter_kind = 0;                 // 0: Lennard-Jones (AIREBO), 1: Morse (AIREBO-M)
    double meps[3], malpha[3], mre[3];  // Morse well depth, stiffness, minimum
};

const std::vector<double>& need(const Params& p, const char* k, size_t n) {
    auto it = p.raw.find(k);
    if (it == p.raw.end() || it->second.size() != n) {
        fprintf(stderr, "oracle: parameter %s missing or of wrong size\n", k);
        throw std::runtime_error(k);
    }
    return it->second;
}

bool parse_params(const char* text, Params& p) {
    std::istringstream in(text);
    std::string line;
    while (std::getline(in, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream ls(line);
        std::string name; size_t n;
        if (!(ls >> name >> n)) continue;
        std::vector<double> v(n);
        for (size_t i = 0; i < n; i++) if (!(ls >> v[i])) return false;
        p.raw[name] = v;
    }
    try {
        auto cp3 = [&](const char* k, double* dst) { auto& v = need(p, k, 3); for (int i = 0; i < 3; i++) dst[i] = v[i]; };
        cp3("Dmin", p.Dmin); cp3("Dmax", p.Dmax); cp3("Q", p.Q); cp3("alpha", p.alpha); cp3("A", p.A);
        double b1[3], b2[3], b3[3], e1[3], e2[3], e3[3];
        cp3("B1", b1); cp3("B2", b2); cp3("B3", b3); cp3("beta1", e1); cp3("beta2", e2); cp3("beta3", e3);
        for (int i = 0; i < 3; i++) {
            p.B[i][0] = b1[i]; p.B[i][1] = b2[i]; p.B[i][2] = b3[i];
            p.beta[i][0] = e1[i]; p.beta[i][1] = e2[i]; p.beta[i][2] = e3[i];
        }
        cp3("rho", p.rho);
        p.lam_coef = need(p, "lambda_coef", 1)[0];
        p.gN0 = need(p, "gC_Nswitch", 2)[0]; p.gN1 = need(p, "gC_Nswitch", 2)[1];
        p.Fx0 = need(p, "Fconj_x", 2)[0]; p.Fx1 = need(p, "Fconj_x", 2)[1];
        p.gC1k = need(p, "gC1.knots", 6); p.gC1d = need(p, "gC1.data", 18);
        p.gC2k = need(p, "gC2.knots", 6); p.gC2d = need(p, "gC2.data", 18);
        p.gHk = need(p, "gH.knots", 4); p.gHd = need(p, "gH.data", 12);
        p.P[0] = need(p, "P.CC", 100); p.P[1] = need(p, "P.CH", 100); p.P[2] = need(p, "P.HC", 100);
        p.piRC[0] = need(p, "piRC.CC", 1800); p.piRC[1] = need(p, "piRC.CH", 1800); p.piRC[2] = need(p, "piRC.HH", 1800);
        p.Tcc = need(p, "Tij.CC", 1800);
        p.guard0 = need(p, "dihedral_guard", 2)[0]; p.guard1 = need(p, "dihedral_guard", 2)[1];
        cp3("lj.sigma", p.sigma); cp3("lj.epsilon", p.eps);
        p.ljcut = need(p, "lj.cut", 1)[0]; p.ljsw = need(p, "lj.switch_start", 1)[0];
        p.SrLo = need(p, "lj.Sr_range", 2)[0]; p.SrHi = need(p, "lj.Sr_range", 2)[1];
        cp3("bstar.bmin", p.bmin); cp3("bstar.bmax", p.bmax); cp3("bstar.rstar", p.rstar);
        cp3("tors.epsilon", p.teps);
        auto it = p.raw.find("inter.kind");
        p.inter_kind = (it != p.raw.end() && it->second.size() == 1) ? (int)it->second[0] : 0;
        if (p.inter_kind == 1) { cp3("morse.epsilon", p.meps); cp3("morse.alpha", p.malpha); cp3("morse.re", p.mre); }
        if (p.inter_kind != 0 && p.inter_kind != 1) return false;
    } catch (...) { return false; }
    return true;
}

// ---------------------------------------------------------------------------
// switching functions and splines, written from their definitions
// ---------------------------------------------------------------------------
// S(t): 1 for t <= 0, 0 for t >= 1, (1 + cos(pi t))/2 in between.
V S(V t) {
    if (t.v <= 0.0) return cst(1.0);
    if (t.v >= 1.0) return cst(0.0);
    return 0.5 * (1.0 + vcos(M_PI * t));
}
// bond weight w_ij(r) = S((r - Dmin)/(Dmax - Dmin))
V wgt(const Params& P, int pij, V r) { return S((r - P.Dmin[pij]) / (P.Dmax[pij] - P.Dmin[pij])); }
// C^1 cubic cut-off of the LJ term: 1 - 3t^2 + 2t^3 on [0,1]
V Sout(V t) {
    if (t.v <= 0.0) return cst(1.0);
    if (t.v >= 1.0) return cst(0.0);
    return 1.0 - t * t * (3.0 - 2.0 * t);
}

// clamp an argument to a spline's domain; a clamped argument carries no derivative
V clampv(V x, double lo, double hi) {
    if (x.v < lo) return cst(lo);
    if (x.v > hi) return cst(hi);
    return x;
}

// quintic Hermite interpolation on knots c_0 < ... < c_m with value, first and
// second derivative given at each knot (data: v, d1, d2 per knot)
V quintic(const std::vector<double>& kn, const std::vector<double>& d, V c) {
    c = clampv(c, kn.front(), kn.back());
    size_t m = 0;
    while (m + 2 < kn.size() && c.v > kn[m + 1]) m++;
    double h = kn[m + 1] - kn[m];
    V t = (c - kn[m]) / h;
    V t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    V H0 = 1.0 - 10.0 * t3 + 15.0 * t4 - 6.0 * t5;
    V H1 = t - 6.0 * t3 + 8.0 * t4 - 3.0 * t5;
    V H2 = 0.5 * t2 - 1.5 * t3 + 1.5 * t4 - 0.5 * t5;
    V H3 = 0.5 * t3 - t4 + 0.5 * t5;
    V H4 = -4.0 * t3 + 7.0 * t4 - 3.0 * t5;
    V H5 = 10.0 * t3 - 15.0 * t4 + 6.0 * t5;
    const double* a = &d[3 * m];
    const double* b = &d[3 * (m + 1)];
    return a[0] * H0 + (h * a[1]) * H1 + (h * h * a[2]) * H2 + (h * h * b[2]) * H3 + (h * b[1]) * H4 + b[0] * H5;
}

// cubic Hermite basis on the unit interval: value basis and slope basis at end e
V hval(V t, int e) { return e == 0 ? 1.0 - t * t * (3.0 - 2.0 * t) : t * t * (3.0 - 2.0 * t); }
V hder(V t, int e) { return e == 0 ? t * (1.0 - t) * (1.0 - t) : t * t * (t - 1.0); }

// bicubic Hermite interpolation on the integer grid [0,4]^2; knot data f, fx, fy, fxy
V bicubic(const std::vector<double>& d, V x, V y) {
    x = clampv(x, 0.0, 4.0); y = clampv(y, 0.0, 4.0);
    int ix = std::min(3, (int)std::floor(x.v)), iy = std::min(3, (int)std::floor(y.v));
    V tx = x - (double)ix, ty = y - (double)iy;
    V sum = cst(0.0);
    for (int ex = 0; ex < 2; ex++)
        for (int ey = 0; ey < 2; ey++) {
            const double* k = &d[((ix + ex) * 5 + (iy + ey)) * 4];
            sum = sum + k[0] * hval(tx, ex) * hval(ty, ey) + k[1] * hder(tx, ex) * hval(ty, ey)
                      + k[2] * hval(tx, ex) * hder(ty, ey) + k[3] * hder(tx, ex) * hder(ty, ey);
        }
    return sum;
}

// tricubic Hermite interpolation (the Lekien-Marsden interpolant) on the integer
// grid [0,4]x[0,4]x[1,9]; knot data f, fx, fy, fz, fxy, fxz, fyz, fxyz
V tricubic(const std::vector<double>& d, V x, V y, V z) {
    x = clampv(x, 0.0, 4.0); y = clampv(y, 0.0, 4.0); z = clampv(z, 1.0, 9.0);
    int ix = std::min(3, (int)std::floor(x.v)), iy = std::min(3, (int)std::floor(y.v));
    int iz = std::min(7, (int)std::floor(z.v - 1.0));
    V tx = x - (double)ix, ty = y - (double)iy, tz = z - 1.0 - (double)iz;
    V sum = cst(0.0);
    for (int ex = 0; ex < 2; ex++)
        for (int ey = 0; ey < 2; ey++)
            for (int ez = 0; ez < 2; ez++) {
                const double* k = &d[(((ix + ex) * 5 + (iy + ey)) * 9 + (iz + ez)) * 8];
                V vx = hval(tx, ex), dx = hder(tx, ex);
                V vy = hval(ty, ey), dy = hder(ty, ey);
                V vz = hval(tz, ez), dz = hder(tz, ez);
                sum = sum + k[0] * vx * vy * vz + k[1] * dx * vy * vz + k[2] * vx * dy * vz
                          + k[3] * vx * vy * dz + k[4] * dx * dy * vz + k[5] * dx * vy * dz
                          + k[6] * vx * dy * dz + k[7] * dx * dy * dz;
            }
    return sum;
}

// ---------------------------------------------------------------------------
// system, neighbour sets with explicit images
// ---------------------------------------------------------------------------
struct Img { int s[3]; };
inline bool same(const Img& a, const Img& b) { return a.s[0] == b.s[0] && a.s[1] == b.s[1] && a.s[2] == b.s[2]; }
inline Img add(const Img& a, const Img& b) { return Img{{a.s[0] + b.s[0], a.s[1] + b.s[1], a.s[2] + b.s[2]}}; }
inline Img neg(const Img& a) { return Img{{-a.s[0], -a.s[1], -a.s[2]}}; }
inline bool positive(const Img& a) {   // lexicographic sign, for self-image pairs
    for (int d = 0; d < 3; d++) { if (a.s[d] > 0) return true; if (a.s[d] < 0) return false; }
    return false;
}

struct Nbr { int j; Img S; };

struct System {
    int64_t n;
    const double* x;       // 3 x n
    const int8_t* t;
    double L[3];
    double pos(int64_t i, int d) const { return x[d * n + i]; }
};

// all (j, S) != (i, 0) with |x_j + S L - x_i| < cutoff(ti, tj), by binning (Sec. 2)
template <class Cut>
void find_pairs(const System& sys, double rmax, Cut cutoff, std::vector<std::vector<Nbr>>& out,
                const char* only = nullptr) {
    int64_t n = sys.n;
    out.assign(n, {});
    int nc[3], m[3];
    for (int d = 0; d < 3; d++) {
        nc[d] = std::max(1, (int)std::floor(sys.L[d] / rmax));
        m[d] = (int)std::ceil(rmax / (sys.L[d] / nc[d]));
    }
    std::vector<int> cell(n), wrap(3 * n);
    std::vector<std::vector<int64_t>> members((size_t)nc[0] * nc[1] * nc[2]);
    for (int64_t i = 0; i < n; i++) {
        int c[3];
        for (int d = 0; d < 3; d++) {
            double xi = sys.pos(i, d);
            int w = (int)std::floor(xi / sys.L[d]);
            double xw = xi - w * sys.L[d];
            c[d] = std::min(nc[d] - 1, std::max(0, (int)std::floor(xw / (sys.L[d] / nc[d]))));
            wrap[3 * i + d] = w;
        }
        cell[i] = (c[0] * nc[1] + c[1]) * nc[2] + c[2];
        members[cell[i]].push_back(i);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        if (only && !only[i]) continue;
        int ci[3] = {cell[i] / (nc[1] * nc[2]), (cell[i] / nc[2]) % nc[1], cell[i] % nc[2]};
        for (int dx = -m[0]; dx <= m[0]; dx++)
            for (int dy = -m[1]; dy <= m[1]; dy++)
                for (int dz = -m[2]; dz <= m[2]; dz++) {
                    int off[3] = {dx, dy, dz}, cc[3], sh[3];
                    for (int d = 0; d < 3; d++) {
                        int q = ci[d] + off[d];
                        int s = (int)std::floor((double)q / nc[d]);
                        cc[d] = q - s * nc[d];
                        sh[d] = s;
                    }
                    int c = (cc[0] * nc[1] + cc[1]) * nc[2] + cc[2];
                    for (int64_t j : members[c]) {
                        Img S;
                        double r2 = 0.0;
                        for (int d = 0; d < 3; d++) {
                            S.s[d] = sh[d] - wrap[3 * j + d] + wrap[3 * i + d];
                            double dd = sys.pos(j, d) + S.s[d] * sys.L[d] - sys.pos(i, d);
                            r2 += dd * dd;
                        }
                        if (j == i && S.s[0] == 0 && S.s[1] == 0 && S.s[2] == 0) continue;
                        double rc = cutoff(sys.t[i], sys.t[j]);
                        if (r2 < rc * rc) out[i].push_back(Nbr{(int)j, S});
                    }
                }
    }
}

// ---------------------------------------------------------------------------
// one term on the tape: leaves keyed by (atom, image relative to the anchor)
// ---------------------------------------------------------------------------
struct TermCtx {
    const System* sys;
    struct Leaf { int64_t atom; Img S; V3 x; };
    std::vector<Leaf> leaves;
    V3 pos(int64_t a, const Img& S) {
        for (auto& l : leaves) if (l.atom == a && same(l.S, S)) return l.x;
        V3 p;
        p.x = leaf(sys->pos(a, 0) + S.s[0] * sys->L[0]);
        p.y = leaf(sys->pos(a, 1) + S.s[1] * sys->L[1]);
        p.z = leaf(sys->pos(a, 2) + S.s[2] * sys->L[2]);
        leaves.push_back(Leaf{a, S, p});
        return p;
    }
};

// accumulates -dE/dx into force arrays and the virial -sum x (x) dE/dx
struct Accum {
    int64_t n;
    double* f;         // 3 x n, may be null
    double W[6];
    const std::vector<char>* sel;   // restrict force accumulation to selected atoms
};

void backprop(TermCtx& T, V E, Accum& acc) {
    if (E.id < 0) { g_tape.clear(); T.leaves.clear(); return; }
    std::vector<double> adj(g_tape.size(), 0.0);
    adj[E.id] = 1.0;
    for (int k = E.id; k >= 0; k--) {
        double a = adj[k];
        if (a == 0.0) continue;
        const Node& nd = g_tape[k];
        if (nd.a >= 0) adj[nd.a] += nd.da * a;
        if (nd.b >= 0) adj[nd.b] += nd.db * a;
    }
    for (auto& l : T.leaves) {
        double g[3] = {l.x.x.id >= 0 ? adj[l.x.x.id] : 0.0, l.x.y.id >= 0 ? adj[l.x.y.id] : 0.0,
                       l.x.z.id >= 0 ? adj[l.x.z.id] : 0.0};
        double p[3] = {l.x.x.v, l.x.y.v, l.x.z.v};
        if (acc.f && (!acc.sel || (*acc.sel)[l.atom]))
            for (int d = 0; d < 3; d++) acc.f[d * acc.n + l.atom] -= g[d];
        acc.W[0] -= p[0] * g[0]; acc.W[1] -= p[1] * g[1]; acc.W[2] -= p[2] * g[2];
        acc.W[3] -= p[0] * g[1]; acc.W[4] -= p[0] * g[2]; acc.W[5] -= p[1] * g[2];
    }
    g_tape.clear();
    T.leaves.clear();
}

// ---------------------------------------------------------------------------
// the potential
// ---------------------------------------------------------------------------
enum Counter { N_BONDS = 0, N_BO_NBR, N_DIHED, N_TORS, N_LJ_CAND, N_LJ_IN, N_LJ_CZERO,
               N_BSTAR, N_BSTAR_DSB, N_PATHS, N_COUNTERS = 16 };

struct Oracle {
    Params P;
    System sys;
    std::vector<std::vector<Nbr>> rebo;   // REBO neighbours, r < Dmax
    std::vector<std::vector<Nbr>> lj;     // LJ half pairs, r < cut * sigma

    int pt(int64_t a, int64_t b) const { return pair_index(sys.t[a], sys.t[b]); }

    // need (nullable): atoms whose REBO neighbours are built; anchor (nullable):
    // atoms whose LJ pairs are built
    void neighbours(const char* need = nullptr, const char* anchor = nullptr) {
        double dmx = 0, rlj = 0;
        for (int p = 0; p < 3; p++) { dmx = std::max(dmx, P.Dmax[p]); rlj = std::max(rlj, P.ljcut * P.sigma[p]); }
        find_pairs(sys, dmx, [&](int a, int b) { return P.Dmax[pair_index(a, b)]; }, rebo, need);
        std::vector<std::vector<Nbr>> full;
        find_pairs(sys, rlj, [&](int a, int b) { return P.ljcut * P.sigma[pair_index(a, b)]; }, full, anchor);
        lj.assign(sys.n, {});
        for (int64_t i = 0; i < sys.n; i++)
            for (auto& nb : full[i])
                if (nb.j > i || (nb.j == i && positive(nb.S))) lj[i].push_back(nb);
    }

    // coordination of atom k: sum of w over all its REBO neighbours (k at image Sk)
    V coordination(TermCtx& T, int64_t k, const Img& Sk, const V3& xk, int64_t skip, const Img& Sskip) {
        V N = cst(0.0);
        for (auto& m : rebo[k]) {
            Img Sm = add(Sk, m.S);
            if (m.j == skip && same(Sm, Sskip)) continue;
            N = N + wgt(P, pt(k, m.j), norm(T.pos(m.j, Sm) - xk));
        }
        return N;
    }

    // p^{sigma pi}_ij for centre c (image Sc) and partner o (image So).  u is the
    // vector used for r_co, umag its length (the true one, or the fictitious
    // constant of b*).  Also returns N_co (total), N^C, N^H of c excluding o.
    V p_sigma_pi(TermCtx& T, int64_t c, const Img& Sc, int64_t o, const Img& So, const V3& u, V umag,
                 V& Ntot, int64_t* cnt) {
        V3 xc = T.pos(c, Sc);
        V NC = cst(0.0), NH = cst(0.0);
        for (auto& k : rebo[c]) {
            Img Sk = add(Sc, k.S);
            if (k.j == o && same(Sk, So)) continue;
            V w = wgt(P, pt(c, k.j), norm(T.pos(k.j, Sk) - xc));
            if (sys.t[k.j] == 0) NC = NC + w; else NH = NH + w;
        }
        Ntot = NC + NH;
        int tc = sys.t[c], to = sys.t[o];
        V sum = cst(0.0);
        for (auto& k : rebo[c]) {
            Img Sk = add(Sc, k.S);
            if (k.j == o && same(Sk, So)) continue;
            V3 rk = T.pos(k.j, Sk) - xc;
            V rkm = norm(rk);
            V w = wgt(P, pt(c, k.j), rkm);
            V cth = clampv(dot(u, rk) / (umag * rkm), -1.0, 1.0);
            V g;
            if (tc == 0) {
                V G = quintic(P.gC1k, P.gC1d, cth);
                V gam = quintic(P.gC2k, P.gC2d, cth);
                V Qn = S((Ntot - P.gN0) / (P.gN1 - P.gN0));
                g = G + Qn * (gam - G);
            } else {
                g = quintic(P.gHk, P.gHd, cth);
            }
            V lam = cst(0.0);
            if (tc == 1) {
                double rho_k = P.rho[pair_index(sys.t[k.j], 1)];
                double rho_o = P.rho[pair_index(to, 1)];
                lam = P.lam_coef * ((rho_k - rkm) - (rho_o - umag));
            }
            sum = sum + w * g * vexp(lam);
            if (cnt) cnt[N_BO_NBR]++;
        }
        V Pij = cst(0.0);
        if (!(tc == 1 && to == 1)) {
            int tab = (tc == 0 && to == 0) ? 0 : (tc == 0 ? 1 : 2);   // CC, CH, HC
            Pij = bicubic(P.P[tab], NC, NH);
        }
        return vpow(1.0 + sum + Pij, -0.5);
    }

    // sum over carbon neighbours k of c (excluding o) of w_ck F(x_ck), x_ck = N_k - w_ck
    V conj_sum(TermCtx& T, int64_t c, const Img& Sc, int64_t o, const Img& So) {
        V3 xc = T.pos(c, Sc);
        V s = cst(0.0);
        for (auto& k : rebo[c]) {
            Img Sk = add(Sc, k.S);
            if (k.j == o && same(Sk, So)) continue;
            if (sys.t[k.j] != 0) continue;
            V3 xk = T.pos(k.j, Sk);
            V w = wgt(P, pt(c, k.j), norm(xk - xc));
            V x = coordination(T, k.j, Sk, xk, c, Sc);
            s = s + w * S((x - P.Fx0) / (P.Fx1 - P.Fx0));
        }
        return s;
    }

    // angle guard of the dihedral sums: 1 unless |cos theta| is within the guard band of 1
    V guard(V c) {
        V a = c.v < 0 ? -c : c;
        return S((a - P.guard0) / P.guard1);
    }

    // b_ij for i (image 0) and j (image Sj); u is the vector standing for r_ij
    V bond_order(TermCtx& T, int64_t i, int64_t j, const Img& Sj, const V3& u, V umag, int64_t* cnt) {
        Img S0{{0, 0, 0}};
        V Nij, Nji;
        V3 mu = {-u.x, -u.y, -u.z};
        V pij = p_sigma_pi(T, i, S0, j, Sj, u, umag, Nij, cnt);
        V pji = p_sigma_pi(T, j, Sj, i, S0, mu, umag, Nji, cnt);
        V A = conj_sum(T, i, S0, j, Sj);
        V B = conj_sum(T, j, Sj, i, S0);
        V Nconj = 1.0 + A * A + B * B;
        int ti = sys.t[i], tj = sys.t[j];
        V pirc;
        if (ti == tj) pirc = tricubic(P.piRC[ti == 0 ? 0 : 2], Nij, Nji, Nconj);
        else if (ti == 0) pirc = tricubic(P.piRC[1], Nij, Nji, Nconj);
        else pirc = tricubic(P.piRC[1], Nji, Nij, Nconj);
        V pidh = cst(0.0);
        if (ti == 0 && tj == 0) {
            V Tij = tricubic(P.Tcc, Nij, Nji, Nconj);
            if (Tij.v != 0.0 || Tij.id >= 0) {
                V3 xi = T.pos(i, S0), xj = T.pos(j, Sj);
                V D = cst(0.0);
                for (auto& k : rebo[i]) {
                    Img Sk = k.S;
                    if (k.j == j && same(Sk, Sj)) continue;
                    V3 rik = T.pos(k.j, Sk) - xi;
                    V rikm = norm(rik);
                    V wik = wgt(P, pt(i, k.j), rikm);
                    V gi = guard(dot(u, rik) / (umag * rikm));
                    if (gi.v == 0.0) continue;
                    for (auto& l : rebo[j]) {
                        Img Sl = add(Sj, l.S);
                        if (l.j == i && same(Sl, S0)) continue;
                        if (l.j == k.j && same(Sl, Sk)) continue;
                        V3 rjl = T.pos(l.j, Sl) - xj;
                        V rjlm = norm(rjl);
                        V wjl = wgt(P, pt(j, l.j), rjlm);
                        V gj = guard(dot(mu, rjl) / (umag * rjlm));
                        if (gj.v == 0.0) continue;
                        V3 n1 = cross(u, rik), n2 = cross(u, rjl);
                        V cw = dot(n1, n2) / (norm(n1) * norm(n2));
                        D = D + (1.0 - cw * cw) * wik * wjl * gi * gj;
                        if (cnt) cnt[N_DIHED]++;
                    }
                }
                pidh = Tij * D;
            }
        }
        return 0.5 * (pij + pji) + pirc + pidh;
    }

    // REBO bond term f_R + b f_A (Alg. 1)
    V rebo_term(TermCtx& T, int64_t i, const Nbr& nb, int64_t* cnt) {
        Img S0{{0, 0, 0}};
        int p = pt(i, nb.j);
        V3 u = T.pos(nb.j, nb.S) - T.pos(i, S0);
        V r = norm(u);
        V w = wgt(P, p, r);
        V fR = w * (1.0 + P.Q[p] / r) * P.A[p] * vexp(-P.alpha[p] * r);
        V fA = cst(0.0);
        for (int m = 0; m < 3; m++)
            if (P.B[p][m] != 0.0) fA = fA - w * P.B[p][m] * vexp(-P.beta[p][m] * r);
        V b = bond_order(T, i, nb.j, nb.S, u, r, cnt);
        if (cnt) cnt[N_BONDS]++;
        return fR + b * fA;
    }

    // torsion around the C-C bond i-j (Alg. 2); omega is the dihedral angle with
    // trans = pi, cos(omega/2)^2 = (1 + cos omega)/2
    V torsion_term(TermCtx& T, int64_t i, const Nbr& nb, int64_t* cnt) {
        Img S0{{0, 0, 0}};
        int64_t j = nb.j;
        const Img& Sj = nb.S;
        V3 xi = T.pos(i, S0), xj = T.pos(j, Sj);
        V3 rij = xj - xi;
        V r = norm(rij);
        V wij = wgt(P, CC, r);
        V3 rji = xi - xj;
        V E = cst(0.0);
        for (auto& k : rebo[i]) {
            Img Sk = k.S;
            if (k.j == j && same(Sk, Sj)) continue;
            V3 rik = T.pos(k.j, Sk) - xi;
            V rikm = norm(rik);
            V wik = wgt(P, pt(i, k.j), rikm);
            V gi = guard(dot(rij, rik) / (r * rikm));
            for (auto& l : rebo[j]) {
                Img Sl = add(Sj, l.S);
                if (l.j == i && same(Sl, S0)) continue;
                if (l.j == k.j && same(Sl, Sk)) continue;
                V3 rjl = T.pos(l.j, Sl) - xj;
                V rjlm = norm(rjl);
                V wjl = wgt(P, pt(j, l.j), rjlm);
                V gj = guard(dot(rji, rjl) / (r * rjlm));
                if (gi.v == 0.0 || gj.v == 0.0) continue;
                V3 n1 = cross(rij, rik), n2 = cross(rij, rjl);
                V cw = dot(n1, n2) / (norm(n1) * norm(n2));
                V half = 0.5 * (1.0 + cw);               // cos^2(omega/2)
                V h5 = half * half * half * half * half;
                double eps = P.teps[(sys.t[k.j] == 1) + (sys.t[l.j] == 1)];
                V Vt = eps * ((256.0 / 405.0) * h5 - 0.1);
                E = E + wik * wij * wjl * gi * gj * Vt;
                if (cnt) cnt[N_TORS]++;
            }
        }
        return E;
    }

    // C_ij search by nested loops (Sec. 4.3): best path from i (image 0) to
    // (j, Sj) over at most three REBO bonds.  Ties: larger weight, then the
    // shorter path, then the smaller (k, l) atom indices.
    struct Path { int len; int64_t k, l; Img Sk, Sl; double w; };
    Path best_path(int64_t i, int64_t j, const Img& Sj) {
        Path best{0, -1, -1, {{0, 0, 0}}, {{0, 0, 0}}, 0.0};
        auto better = [&](const Path& c) {
            if (c.w != best.w) return c.w > best.w;
            if (c.len != best.len) return c.len < best.len;
            if (c.k != best.k) return c.k < best.k;
            return c.l < best.l;
        };
        auto wnum = [&](int64_t a, const Img& Sa, int64_t b, const Img& Sb) {
            double r2 = 0;
            for (int d = 0; d < 3; d++) {
                double dd = sys.pos(b, d) + Sb.s[d] * sys.L[d] - sys.pos(a, d) - Sa.s[d] * sys.L[d];
                r2 += dd * dd;
            }
            return wgt(P, pt(a, b), cst(std::sqrt(r2))).v;
        };
        Img S0{{0, 0, 0}};
        for (auto& k : rebo[i]) {
            if (k.j == j && same(k.S, Sj)) {
                Path c{1, -1, -1, S0, S0, wnum(i, S0, j, Sj)};
                if (better(c)) best = c;
                continue;
            }
            if (k.j == i) continue;
            double wik = wnum(i, S0, k.j, k.S);
            for (auto& l : rebo[k.j]) {
                Img Sl = add(k.S, l.S);
                if (l.j == i && same(Sl, S0)) continue;
                if (l.j == j && same(Sl, Sj)) {
                    Path c{2, k.j, -1, k.S, S0, wik * wnum(k.j, k.S, j, Sj)};
                    if (better(c)) best = c;
                    continue;
                }
                double wkl = wnum(k.j, k.S, l.j, Sl);
                for (auto& m : rebo[l.j]) {
                    Img Sm = add(Sl, m.S);
                    if (m.j == j && same(Sm, Sj)) {
                        Path c{3, k.j, l.j, k.S, Sl, wik * wkl * wnum(l.j, Sl, j, Sj)};
                        if (better(c)) best = c;
                    }
                }
            }
        }
        return best;
    }

    // LJ pair term (Alg. 3) for i (image 0) and (j, Sj)
    V lj_term(TermCtx& T, int64_t i, const Nbr& nb, int64_t* cnt, bool* dsb_nonzero) {
        Img S0{{0, 0, 0}};
        int p = pt(i, nb.j);
        Path path = best_path(i, nb.j, nb.S);
        if (cnt) cnt[N_LJ_IN]++;
        if (path.w >= 1.0) { if (cnt) cnt[N_LJ_CZERO]++; return cst(0.0); }
        V3 xi = T.pos(i, S0), xj = T.pos(nb.j, nb.S);
        V3 d = xj - xi;
        V r = norm(d);
        V wmax = cst(0.0);
        if (path.len == 1) wmax = wgt(P, p, r);
        else if (path.len == 2) {
            V3 xk = T.pos(path.k, path.Sk);
            wmax = wgt(P, pt(i, path.k), norm(xk - xi)) * wgt(P, pt(path.k, nb.j), norm(xj - xk));
        } else if (path.len == 3) {
            V3 xk = T.pos(path.k, path.Sk), xl = T.pos(path.l, path.Sl);
            wmax = wgt(P, pt(i, path.k), norm(xk - xi)) * wgt(P, pt(path.k, path.l), norm(xl - xk))
                 * wgt(P, pt(path.l, nb.j), norm(xj - xl));
        }
        V C = 1.0 - wmax;
        double sg = P.sigma[p];
        V sr = sg / r;
        V sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
        V VLJ = 4.0 * P.eps[p] * (sr6 * sr6 - sr6);
        if (P.inter_kind == 1) {      // AIREBO-M: Morse in place of Lennard-Jones (Sec. 2.1.2)
            V e = vexp(-P.malpha[p] * (r - P.mre[p]));
            VLJ = P.meps[p] * (e * e - 2.0 * e);
        }
        VLJ = VLJ * Sout((r - P.ljsw * sg) / ((P.ljcut - P.ljsw) * sg));
        V Sr = S((r - P.SrLo * sg) / ((P.SrHi - P.SrLo) * sg));
        V factor = cst(1.0);
        if (Sr.v > 0.0) {
            double rs = P.rstar[p];
            V3 u = d * (rs / r);
            V bstar = bond_order(T, i, nb.j, nb.S, u, cst(rs), nullptr);
            V Sb = S((bstar - P.bmin[p]) / (P.bmax[p] - P.bmin[p]));
            factor = Sr * Sb + 1.0 - Sr;
            if (cnt) cnt[N_BSTAR]++;
            if (Sb.id >= 0 && dsb_nonzero) *dsb_nonzero = true;
        }
        return factor * C * VLJ;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// C ABI for the tests (ctypes)
// ---------------------------------------------------------------------------
extern "C" {

void* oracle_create(const char* param_text) {
    Oracle* o = new Oracle();
    if (!parse_params(param_text, o->P)) { delete o; return nullptr; }
    return o;
}

void oracle_destroy(void* h) { delete (Oracle*)h; }

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// flags: bit0 REBO, bit1 LJ, bit2 torsion.
// sel (nullable): per-atom 0/1 mask.  With a mask only the terms anchored at
// atoms flagged in `anchor` are evaluated and only selected atoms get forces.
// energy4 = total, REBO, LJ, torsion (over the evaluated terms).
// need (nullable): atoms whose REBO neighbour sets are needed by the anchored
// terms (all atoms when null).
// eatom (nullable, n doubles): per-atom energies, each term (a REBO bond, the
// torsion term of a C-C bond, an LJ pair) split evenly between the two atoms
// i and j that define it.
int oracle_compute_masked(void* h, int64_t n, const double* pos, const int8_t* types, const double* box,
                          int flags, const char* anchor, const char* sel, const char* need, double* force,
                          double* energy4, double* virial6, int64_t* counters, double* eatom) {
    Oracle* o = (Oracle*)h;
    o->sys.n = n; o->sys.x = pos; o->sys.t = types;
    for (int d = 0; d < 3; d++) o->sys.L[d] = box[d];
    o->neighbours(need, anchor);
    std::vector<char> selv;
    if (sel) selv.assign(sel, sel + n);
    if (force) std::fill(force, force + 3 * n, 0.0);
    if (eatom) std::fill(eatom, eatom + n, 0.0);
    double E[4] = {0, 0, 0, 0}, W[6] = {0, 0, 0, 0, 0, 0};
    int64_t cnt[N_COUNTERS] = {0};
    int nthr = oracle_threads();
    std::vector<std::vector<double>> fthr(nthr, std::vector<double>(force ? 3 * n : 0, 0.0));
    std::vector<std::vector<double>> ethr(nthr, std::vector<double>(eatom ? n : 0, 0.0));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        Accum acc{n, force ? fthr[tid].data() : nullptr, {0, 0, 0, 0, 0, 0}, sel ? &selv : nullptr};
        double Et[4] = {0, 0, 0, 0};
        int64_t ct[N_COUNTERS] = {0};
        TermCtx T; T.sys = &o->sys;
        double* ea = eatom ? ethr[tid].data() : nullptr;
        auto split = [&](int64_t a, int64_t b, double e) {
            if (ea) { ea[a] += 0.5 * e; ea[b] += 0.5 * e; }
        };
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; i++) {
            if (anchor && !anchor[i]) continue;
            if (flags & 1)
                for (auto& nb : o->rebo[i]) {
                    if (nb.j <= i) continue;
                    V e = o->rebo_term(T, i, nb, ct);
                    Et[1] += e.v;
                    split(i, nb.j, e.v);
                    backprop(T, e, acc);
                }
            if (flags & 4)
                for (auto& nb : o->rebo[i]) {
                    if (nb.j <= i || types[i] != 0 || types[nb.j] != 0) continue;
                    V e = o->torsion_term(T, i, nb, ct);
                    Et[3] += e.v;
                    split(i, nb.j, e.v);
                    backprop(T, e, acc);
                }
            if (flags & 2)
                for (auto& nb : o->lj[i]) {
                    bool dsb = false;
                    V e = o->lj_term(T, i, nb, ct, &dsb);
                    if (dsb) ct[N_BSTAR_DSB]++;
                    Et[2] += e.v;
                    split(i, nb.j, e.v);
                    backprop(T, e, acc);
                }
        }
#pragma omp critical
        {
            for (int k = 0; k < 4; k++) E[k] += Et[k];
            for (int k = 0; k < 6; k++) W[k] += acc.W[k];
            for (int k = 0; k < N_COUNTERS; k++) cnt[k] += ct[k];
        }
    }
    if (force)
        for (int t = 0; t < nthr; t++)
            for (int64_t k = 0; k < 3 * n; k++) force[k] += fthr[t][k];
    if (eatom)
        for (int t = 0; t < nthr; t++)
            for (int64_t k = 0; k < n; k++) eatom[k] += ethr[t][k];
    E[0] = E[1] + E[2] + E[3];
    if (energy4) for (int k = 0; k < 4; k++) energy4[k] = E[k];
    if (virial6) for (int k = 0; k < 6; k++) virial6[k] = W[k];
    for (int64_t i = 0; i < n; i++) cnt[N_LJ_CAND] += (int64_t)o->lj[i].size();
    if (counters) for (int k = 0; k < N_COUNTERS; k++) counters[k] = cnt[k];
    return 0;
}

int oracle_compute(void* h, int64_t n, const double* pos, const int8_t* types, const double* box, int flags,
                   double* force, double* energy4, double* virial6, int64_t* counters, double* eatom) {
    return oracle_compute_masked(h, n, pos, types, box, flags, nullptr, nullptr, nullptr, force, energy4, virial6,
                                 counters, eatom);
}

// REBO neighbour sets (r < Dmax) as flat arrays; returns the total count, or
// -1 if cap is too small.  offsets has n+1 entries.
int64_t oracle_rebo_neighbors(void* h, int64_t n, const double* pos, const int8_t* types, const double* box,
                              int64_t cap, int32_t* out_j, int8_t* out_img, int64_t* offsets) {
    Oracle* o = (Oracle*)h;
    o->sys.n = n; o->sys.x = pos; o->sys.t = types;
    for (int d = 0; d < 3; d++) o->sys.L[d] = box[d];
    o->neighbours();
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        offsets[i] = c;
        for (auto& nb : o->rebo[i]) {
            if (c >= cap) return -1;
            out_j[c] = nb.j;
            for (int d = 0; d < 3; d++) out_img[3 * c + d] = (int8_t)nb.S.s[d];
            c++;
        }
    }
    offsets[n] = c;
    return c;
}

// LJ half-pair sets (r < cut sigma_ij), same layout
int64_t oracle_lj_pairs(void* h, int64_t n, const double* pos, const int8_t* types, const double* box,
                        int64_t cap, int32_t* out_j, int8_t* out_img, int64_t* offsets) {
    Oracle* o = (Oracle*)h;
    o->sys.n = n; o->sys.x = pos; o->sys.t = types;
    for (int d = 0; d < 3; d++) o->sys.L[d] = box[d];
    o->neighbours();
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) {
        offsets[i] = c;
        for (auto& nb : o->lj[i]) {
            if (c >= cap) return -1;
            out_j[c] = nb.j;
            for (int d = 0; d < 3; d++) out_img[3 * c + d] = (int8_t)nb.S.s[d];
            c++;
        }
    }
    offsets[n] = c;
    return c;
}

// C_ij of one pair (after oracle_rebo_neighbors / oracle_compute set up the system)
double oracle_cij(void* h, int64_t i, int64_t j, const int32_t* img, int32_t* path_out) {
    Oracle* o = (Oracle*)h;
    Img S{{img[0], img[1], img[2]}};
    auto p = o->best_path(i, j, S);
    if (path_out) { path_out[0] = p.len; path_out[1] = (int32_t)p.k; path_out[2] = (int32_t)p.l; }
    return 1.0 - p.w;
}

// spline and switch evaluation for the pins.  which: 0 gC1, 1 gC2, 2 gH,
// 10..12 P (CC, CH, HC), 20..22 pi^rc (CC, CH, HH), 30 T_CC, 40 S, 41 Sout.
// Returns the value, writes the gradient w.r.t. (x, y, z) to grad.
double oracle_spline(void* h, int which, double x, double y, double z, double* grad) {
    Oracle* o = (Oracle*)h;
    g_tape.clear();
    V X = leaf(x), Y = leaf(y), Z = leaf(z);
    V r;
    const Params& P = o->P;
    if (which == 0) r = quintic(P.gC1k, P.gC1d, X);
    else if (which == 1) r = quintic(P.gC2k, P.gC2d, X);
    else if (which == 2) r = quintic(P.gHk, P.gHd, X);
    else if (which >= 10 && which <= 12) r = bicubic(P.P[which - 10], X, Y);
    else if (which >= 20 && which <= 22) r = tricubic(P.piRC[which - 20], X, Y, Z);
    else if (which == 30) r = tricubic(P.Tcc, X, Y, Z);
    else if (which == 40) r = S(X);
    else if (which == 41) r = Sout(X);
    else return NAN;
    std::vector<double> adj(g_tape.size(), 0.0);
    if (r.id >= 0) {
        adj[r.id] = 1.0;
        for (int k = r.id; k >= 0; k--) {
            const Node& nd = g_tape[k];
            if (nd.a >= 0) adj[nd.a] += nd.da * adj[k];
            if (nd.b >= 0) adj[nd.b] += nd.db * adj[k];
        }
    }
    if (grad) { grad[0] = adj[X.id]; grad[1] = adj[Y.id]; grad[2] = adj[Z.id]; }
    g_tape.clear();
    return r.v;
}

}  // extern "C"
