// Host construction of the site orderings and neighbour tables (see geometry.h).
#include <cuda_fp16.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <string>
#include <unordered_map>

#include "geometry.h"

namespace dwf {

namespace {

inline long lexi(const int *L, const int *x)
{
    return x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
}
inline int pad_to(int n, int m) { return (n + m - 1) / m * m; }

// Neighbour entry: input index with the boundary sign folded in.
inline int enc(long idx, bool neg) { return neg ? (int)(-idx - 2) : (int)idx; }

// Does the hop from global coordinate x in direction mu, dir cross the
// antiperiodic t boundary?
inline bool crosses_t(const LatticeGeom &g, const int *x, int mu, int dir)
{
    if (!g.antiperiodic_t || mu != 3) return false;
    return dir > 0 ? x[3] == g.L[3] - 1 : x[3] == 0;
}

// Link source for output site x, direction k = 2 mu + d (d = 0: +mu, 1: -mu):
// forward U_{x,mu}; backward U^+_{x-mu,mu}.
inline long link_src(const LatticeGeom &g, const int *x, int mu, int d)
{
    int y[4] = {x[0], x[1], x[2], x[3]};
    if (d == 0) return (lexi(g.L, y) * 4 + mu) * 2 + 0;
    y[mu] = (y[mu] - 1 + g.L[mu]) % g.L[mu];
    return (lexi(g.L, y) * 4 + mu) * 2 + 1;
}

struct RelKeyHash {
    size_t operator()(long k) const { return std::hash<long>()(k); }
};

}  // namespace

bool build_geometry(LatticeGeom &g, const int dims[4], const int subd[4], int anti, std::string &err)
{
    for (int mu = 0; mu < 4; mu++) {
        g.L[mu] = dims[mu];
        g.sub[mu] = subd ? subd[mu] : dims[mu];
        if (g.L[mu] <= 0 || g.L[mu] % 2) {
            err = "lattice extents must be positive and even";
            return false;
        }
        if (g.sub[mu] <= 0 || g.sub[mu] % 2 || g.L[mu] % g.sub[mu]) {
            err = "block extents must be even and divide the lattice extents";
            return false;
        }
        if (g.sub[mu] != g.L[mu] && g.L[mu] - g.sub[mu] < 4) {
            err = "a partitioned dimension needs lattice - block extent >= 4";
            return false;
        }
        g.nbk[mu] = g.L[mu] / g.sub[mu];
    }
    g.antiperiodic_t = anti != 0;
    g.V = (long)g.L[0] * g.L[1] * g.L[2] * g.L[3];
    g.Vh = g.V / 2;
    g.nblk = g.nbk[0] * g.nbk[1] * g.nbk[2] * g.nbk[3];
    const long bvol = (long)g.sub[0] * g.sub[1] * g.sub[2] * g.sub[3];
    g.Nb = (int)(bvol / 2);
    g.Nb_pad = pad_to(g.Nb, kSegPad);

    bool part[4];
    for (int mu = 0; mu < 4; mu++) part[mu] = g.sub[mu] != g.L[mu];

    // relative coordinates r of the extended region, r_mu in [-2, sub+1] for
    // partitioned dims, [0, sub-1] otherwise
    int lo[4], ext[4];
    for (int mu = 0; mu < 4; mu++) {
        lo[mu] = part[mu] ? -2 : 0;
        ext[mu] = part[mu] ? g.sub[mu] + 4 : g.sub[mu];
    }
    auto rkey = [&](const int *r) {
        return (long)(r[0] - lo[0]) +
               (long)ext[0] * ((r[1] - lo[1]) + (long)ext[1] * ((r[2] - lo[2]) + (long)ext[2] * (r[3] - lo[3])));
    };
    auto dist = [&](const int *r) {
        int d = 0;
        for (int mu = 0; mu < 4; mu++) {
            if (!part[mu]) continue;
            if (r[mu] < 0) d += -r[mu];
            else if (r[mu] >= g.sub[mu]) d += r[mu] - g.sub[mu] + 1;
        }
        return d;
    };
    // enumerate region sites
    std::vector<std::array<int, 4>> interior, o1, e2_halo1, e2_halo2;
    {
        int r[4];
        for (r[3] = lo[3]; r[3] < lo[3] + ext[3]; r[3]++)
            for (r[2] = lo[2]; r[2] < lo[2] + ext[2]; r[2]++)
                for (r[1] = lo[1]; r[1] < lo[1] + ext[1]; r[1]++)
                    for (r[0] = lo[0]; r[0] < lo[0] + ext[0]; r[0]++) {
                        const int d = dist(r);
                        const int par = ((r[0] + r[1] + r[2] + r[3]) % 2 + 2) % 2;
                        std::array<int, 4> a = {r[0], r[1], r[2], r[3]};
                        if (par == 0) {
                            if (d == 0) interior.push_back(a);
                            else if (d == 1) e2_halo1.push_back(a);
                            else if (d == 2) e2_halo2.push_back(a);
                        } else if (d <= 1) {
                            o1.push_back(a);
                        }
                    }
        // odd interior first inside O1
        std::stable_partition(o1.begin(), o1.end(), [&](const std::array<int, 4> &a) {
            return dist(a.data()) == 0;
        });
    }
    // Halo sites have only some of their eight neighbours in the input region
    // of the stage that writes them (stage 1 for O1: the interior; stage 2 for
    // E2: O1).  Ordering each halo by that neighbour pattern keeps the sites
    // of a warp on the same directions (no divergence in the hop).
    {
        auto pattern = [&](const std::array<int, 4> &a, int maxd) {
            int m = 0;
            for (int mu = 0; mu < 4; mu++)
                for (int d = 0; d < 2; d++) {
                    int n[4] = {a[0], a[1], a[2], a[3]};
                    n[mu] += d ? -1 : 1;
                    if (!part[mu]) n[mu] = (n[mu] + g.sub[mu]) % g.sub[mu];
                    if (dist(n) <= maxd) m |= 1 << (2 * mu + d);
                }
            return m;
        };
        auto by_pattern = [&](std::vector<std::array<int, 4>>::iterator b,
                              std::vector<std::array<int, 4>>::iterator e, int maxd) {
            std::vector<std::pair<int, std::array<int, 4>>> tmp;
            for (auto it = b; it != e; ++it) tmp.push_back({pattern(*it, maxd), *it});
            std::stable_sort(tmp.begin(), tmp.end(),
                             [](const auto &x, const auto &y) { return x.first < y.first; });
            for (auto &t : tmp) *b++ = t.second;
        };
        auto ob = std::find_if(o1.begin(), o1.end(),
                               [&](const std::array<int, 4> &a) { return dist(a.data()) != 0; });
        by_pattern(ob, o1.end(), 0);
        e2_halo1.insert(e2_halo1.end(), e2_halo2.begin(), e2_halo2.end());
        e2_halo2.clear();
        by_pattern(e2_halo1.begin(), e2_halo1.end(), 1);
    }
    if ((int)interior.size() != g.Nb) {
        err = "internal: interior count mismatch";
        return false;
    }
    g.O1 = (int)o1.size();
    g.O1_pad = pad_to(g.O1, kSegPad);
    g.E2 = g.Nb_pad + (int)(e2_halo1.size() + e2_halo2.size());
    g.E2_pad = pad_to(g.E2, kSegPad);

    std::unordered_map<long, int> idx_int, idx_o1, idx_e2;
    for (int k = 0; k < (int)interior.size(); k++) {
        idx_int[rkey(interior[k].data())] = k;
        idx_e2[rkey(interior[k].data())] = k;
    }
    for (int k = 0; k < (int)o1.size(); k++) idx_o1[rkey(o1[k].data())] = k;
    {
        int k = g.Nb_pad;
        for (auto &a : e2_halo1) idx_e2[rkey(a.data())] = k++;
        for (auto &a : e2_halo2) idx_e2[rkey(a.data())] = k++;
    }
    // E2 list in index order (with padding holes)
    std::vector<std::array<int, 4>> e2list(g.E2_pad, {{1 << 20, 0, 0, 0}});
    for (int k = 0; k < (int)interior.size(); k++) e2list[k] = interior[k];
    {
        int k = g.Nb_pad;
        for (auto &a : e2_halo1) e2list[k++] = a;
        for (auto &a : e2_halo2) e2list[k++] = a;
    }

    // ------------------------------------------------ packed global orders
    const long ne = g.ne();
    g.even_cb.assign(ne, -1);
    g.odd_cb.assign(ne, -1);
    std::vector<long> packed_of_lex(g.V, -1);
    // odd interior of a block: odd sites with d = 0, in O1 order (first entries)
    for (int b = 0; b < g.nblk; b++) {
        int bc[4], rem = b;
        for (int mu = 0; mu < 4; mu++) {
            bc[mu] = rem % g.nbk[mu];
            rem /= g.nbk[mu];
        }
        int oi = 0;
        for (int k = 0; k < (int)interior.size(); k++) {
            int x[4];
            for (int mu = 0; mu < 4; mu++) x[mu] = bc[mu] * g.sub[mu] + interior[k][mu];
            const long lex = lexi(g.L, x);
            g.even_cb[(long)b * g.Nb_pad + k] = lex / 2;
            packed_of_lex[lex] = (long)b * g.Nb_pad + k;
        }
        for (int k = 0; k < (int)o1.size(); k++) {
            if (dist(o1[k].data()) != 0) break;
            int x[4];
            for (int mu = 0; mu < 4; mu++) x[mu] = bc[mu] * g.sub[mu] + o1[k][mu];
            const long lex = lexi(g.L, x);
            g.odd_cb[(long)b * g.Nb_pad + oi] = lex / 2;
            packed_of_lex[lex] = (long)b * g.Nb_pad + oi;
            oi++;
        }
        if (oi != g.Nb) {
            err = "internal: odd interior count mismatch";
            return false;
        }
    }

    // global tables
    auto global_tables = [&](const std::vector<long> &cb_of, int par, std::vector<int> &nbr,
                             std::vector<long> &lnk) {
        nbr.assign(ne * 8, -1);
        lnk.assign(ne * 8, -1);
        for (long i = 0; i < ne; i++) {
            const long cb = cb_of[i];
            if (cb < 0) continue;
            // recover coordinates: lex = 2 cb + offset
            long lex = 2 * cb;
            int x[4];
            {
                long t = lex;
                x[0] = (int)(t % g.L[0]); t /= g.L[0];
                x[1] = (int)(t % g.L[1]); t /= g.L[1];
                x[2] = (int)(t % g.L[2]);
                x[3] = (int)(t / g.L[2]);
            }
            if (((x[0] + x[1] + x[2] + x[3]) & 1) != par) {
                x[0] += 1;
            }
            for (int mu = 0; mu < 4; mu++)
                for (int d = 0; d < 2; d++) {
                    const int dir = d ? -1 : 1;
                    int y[4] = {x[0], x[1], x[2], x[3]};
                    y[mu] = (y[mu] + dir + g.L[mu]) % g.L[mu];
                    const long nl = lexi(g.L, y);
                    nbr[i * 8 + 2 * mu + d] = enc(packed_of_lex[nl], crosses_t(g, x, mu, dir));
                    lnk[i * 8 + 2 * mu + d] = link_src(g, x, mu, d);
                }
        }
    };
    global_tables(g.even_cb, 0, g.nbr_e, g.lnk_e);
    global_tables(g.odd_cb, 1, g.nbr_o, g.lnk_o);

    // ------------------------------------------------ local tables
    const long nO1 = (long)g.nblk * g.O1_pad, nE2 = (long)g.nblk * g.E2_pad;
    const long nI = (long)g.nblk * g.Nb_pad;
    g.t1.assign(nO1 * 8, -1);
    g.t3.assign(nO1 * 8, -1);
    g.t2.assign(nE2 * 8, -1);
    g.t4.assign(nI * 8, -1);
    g.lnk_O1.assign(nO1 * 8, -1);
    g.lnk_E2.assign(nE2 * 8, -1);
    for (int b = 0; b < g.nblk; b++) {
        int bc[4], rem = b;
        for (int mu = 0; mu < 4; mu++) {
            bc[mu] = rem % g.nbk[mu];
            rem /= g.nbk[mu];
        }
        auto global_x = [&](const int *r, int *x) {
            for (int mu = 0; mu < 4; mu++) x[mu] = ((bc[mu] * g.sub[mu] + r[mu]) % g.L[mu] + g.L[mu]) % g.L[mu];
        };
        auto step = [&](const int *r, int mu, int dir, int *n) {
            for (int m = 0; m < 4; m++) n[m] = r[m];
            n[mu] += dir;
            if (!part[mu]) n[mu] = (n[mu] + g.sub[mu]) % g.sub[mu];
        };
        // O1 outputs: t1 (-> interior), t3 (-> E2)
        for (int k = 0; k < (int)o1.size(); k++) {
            const long row = (long)b * g.O1_pad + k;
            int x[4];
            global_x(o1[k].data(), x);
            for (int mu = 0; mu < 4; mu++)
                for (int d = 0; d < 2; d++) {
                    const int dir = d ? -1 : 1;
                    int n[4];
                    step(o1[k].data(), mu, dir, n);
                    const bool neg = crosses_t(g, x, mu, dir);
                    g.lnk_O1[row * 8 + 2 * mu + d] = link_src(g, x, mu, d);
                    const long key = rkey(n);
                    bool inbox = true;
                    for (int m = 0; m < 4; m++)
                        if (n[m] < lo[m] || n[m] >= lo[m] + ext[m]) inbox = false;
                    if (!inbox) {
                        err = "internal: O1 neighbour outside the extended box";
                        return false;
                    }
                    auto it = idx_int.find(key);
                    if (it != idx_int.end()) g.t1[row * 8 + 2 * mu + d] = enc((long)b * g.Nb_pad + it->second, neg);
                    auto je = idx_e2.find(key);
                    if (je == idx_e2.end()) {
                        err = "internal: O1 neighbour missing from E2";
                        return false;
                    }
                    g.t3[row * 8 + 2 * mu + d] = enc((long)b * g.E2_pad + je->second, neg);
                }
        }
        // E2 outputs: t2 (-> O1); interior rows also give t4
        for (int k = 0; k < g.E2_pad; k++) {
            if (e2list[k][0] == (1 << 20)) continue;
            const long row = (long)b * g.E2_pad + k;
            int x[4];
            global_x(e2list[k].data(), x);
            for (int mu = 0; mu < 4; mu++)
                for (int d = 0; d < 2; d++) {
                    const int dir = d ? -1 : 1;
                    int n[4];
                    step(e2list[k].data(), mu, dir, n);
                    const bool neg = crosses_t(g, x, mu, dir);
                    g.lnk_E2[row * 8 + 2 * mu + d] = link_src(g, x, mu, d);
                    bool inbox = true;
                    for (int m = 0; m < 4; m++)
                        if (n[m] < lo[m] || n[m] >= lo[m] + ext[m]) inbox = false;
                    if (!inbox) continue;
                    auto it = idx_o1.find(rkey(n));
                    if (it == idx_o1.end()) continue;
                    g.t2[row * 8 + 2 * mu + d] = enc((long)b * g.O1_pad + it->second, neg);
                    if (k < g.Nb) g.t4[((long)b * g.Nb_pad + k) * 8 + 2 * mu + d] = enc((long)b * g.O1_pad + it->second, neg);
                }
            if (k < g.Nb)
                for (int j = 0; j < 8; j++)
                    if (g.t4[((long)b * g.Nb_pad + k) * 8 + j] == -1) {
                        err = "internal: interior neighbour missing from O1";
                        return false;
                    }
        }
    }
    return true;
}

void gather_links(const std::vector<long> &src, const double *gauge, Prec p,
                  std::vector<unsigned char> &out)
{
    const size_t n = src.size();
    const int eb = p == P64 ? 8 : p == P32 ? 4 : 2;
    out.assign(n * 12 * eb, 0);
    for (size_t e = 0; e < n; e++) {
        if (src[e] < 0) continue;
        const long link = src[e] >> 1;
        const bool dag = src[e] & 1;
        const double *U = gauge + link * 18;  // 3x3 complex
        double m[12];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) {
                // dagger: (U^+)_{rc} = conj(U_{cr})
                const double re = dag ? U[(c * 3 + r) * 2] : U[(r * 3 + c) * 2];
                const double im = dag ? -U[(c * 3 + r) * 2 + 1] : U[(r * 3 + c) * 2 + 1];
                m[(r * 3 + c) * 2] = re;
                m[(r * 3 + c) * 2 + 1] = im;
            }
        unsigned char *dst = out.data() + e * 12 * eb;
        for (int q = 0; q < 12; q++) {
            if (p == P64) {
                std::memcpy(dst + q * 8, &m[q], 8);
            } else if (p == P32) {
                float f = (float)m[q];
                std::memcpy(dst + q * 4, &f, 4);
            } else {
                __half h = __float2half_rn((float)m[q]);
                std::memcpy(dst + q * 2, &h, 2);
            }
        }
    }
}

}  // namespace dwf
