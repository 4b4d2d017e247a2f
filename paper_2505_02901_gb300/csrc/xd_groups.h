// xd_groups.h -- host-side questions about a bond list under a group of site
// permutations (Sec. 3.9-3.10): which bonds lie on one orbit, and whether the
// couplings are invariant.  Plain C++ without CUDA; bonds are [nb][2] site
// pairs, perms [G][N] with perms[g][i] = g(i).  A hash of the unordered site
// pair turns each question into G x nb lookups.
#pragma once

#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

namespace xd {

class PairIndex {
  public:
    PairIndex(const int32_t *bonds, int nb) {
        for (int k = 0; k < nb; ++k) map_[key(bonds[2 * k], bonds[2 * k + 1])].push_back(k);
    }
    // bonds on the site pair {i, j}, or nullptr
    const std::vector<int> *find(int i, int j) const {
        auto it = map_.find(key(i, j));
        return it == map_.end() ? nullptr : &it->second;
    }

  private:
    static uint64_t key(int i, int j) {
        const uint32_t a = (uint32_t)(i < j ? i : j), b = (uint32_t)(i < j ? j : i);
        return ((uint64_t)a << 32) | b;
    }
    std::unordered_map<uint64_t, std::vector<int>> map_;
};

// orb[p] = orbit id of bond p: bonds share an id when some g maps the site
// pair of one onto the site pair of the other; ids are numbered in the order
// of each orbit's first bond.  Returns the number of orbits.
inline int bond_orbits(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, int32_t *orb) {
    const PairIndex idx(bonds, nb);
    for (int p = 0; p < nb; ++p) orb[p] = -1;
    int norb = 0;
    for (int q = 0; q < nb; ++q) {
        if (orb[q] >= 0) continue;
        for (int g = 0; g < G; ++g) {
            const int32_t *pg = perms + (size_t)g * N;
            const std::vector<int> *hit = idx.find(pg[bonds[2 * q]], pg[bonds[2 * q + 1]]);
            if (hit)
                for (int p : *hit)
                    if (orb[p] < 0) orb[p] = norb;
        }
        ++norb;
    }
    return norb;
}

// 1 when the image of every bond under every g is a bond with the same
// coupling; else 0, with the first failing (g, k) in g-major order.
inline int couplings_invariant(int N, int G, const int32_t *perms, const int32_t *bonds, int nb,
                               const double *J, int *bad_g, int *bad_k) {
    const PairIndex idx(bonds, nb);
    for (int g = 0; g < G; ++g) {
        const int32_t *pg = perms + (size_t)g * N;
        for (int k = 0; k < nb; ++k) {
            const std::vector<int> *hit = idx.find(pg[bonds[2 * k]], pg[bonds[2 * k + 1]]);
            bool ok = false;
            if (hit)
                for (int q : *hit)
                    if (J[q] == J[k]) {
                        ok = true;
                        break;
                    }
            if (!ok) {
                *bad_g = g;
                *bad_k = k;
                return 0;
            }
        }
    }
    return 1;
}

// Tables for the orbit search of a symmetric block (Sec. 3.10): the byte
// tables of the action, and the fast searches that apply to the group.
//   act[(g nchunk + c) 256 + v] = g applied to the bits v << 8c, where g acts
//   on a state word by (g s)_i = s_{g(i)}.
//   Torus: the group holds every translation T_{a,b} of an Lx x Ly torus
//   (site x + Lx y, 2 <= Lx <= 8).  It is the union of the cosets
//   {s -> T_{a,b}(p_k s)}, p_0 the identity: tpp[k] = group index of p_k,
//   tg[k Lx Ly + a + Lx b] = group index of s -> T_{a,b}(p_k s), whose site
//   map is i -> p_k(T_{a,b}(i)); tnp = number of cosets, 0 when only the
//   translations; minrot[r] / amask[r] = smallest rotation of an Lx-bit row
//   and the rotations reaching it; cut (Lx <= 7) = the same over a subset of
//   the rotations (xd_orbit.h); pm[(k - 1) nb + q] = p_k applied to the
//   mask of bond q (k >= 1).
//   Ring (only without a torus): the group is the N rotations i -> i + n,
//   with or without the N reflections i -> n - i (mod N); cg[n] and
//   cg[N + n] are their group indices, cdih = 1 with reflections.
struct GroupTables {
    int nchunk = 0;
    std::vector<uint64_t> act;
    int tx = 0, ty = 0, tnp = 0;
    std::vector<uint8_t> minrot, amask;
    std::vector<uint16_t> cut;  // Lx <= 7: cut[(r << Lx) | A] (xd_orbit.h)
    std::vector<int16_t> tg, tpp;
    std::vector<uint64_t> pm;
    int cn = 0, cdih = 0;
    std::vector<int16_t> cg;
};

inline void group_tables(int N, int G, const int32_t *perms, const int32_t *bonds, int nb, GroupTables *out) {
    GroupTables &T = *out;
    auto perm = [&](int g) { return perms + (size_t)g * N; };
    T.nchunk = (N + 7) / 8;
    T.act.assign((size_t)G * T.nchunk * 256, 0);
    std::vector<int> inv(N);
    for (int g = 0; g < G; ++g) {
        for (int i = 0; i < N; ++i) inv[perm(g)[i]] = i;  // bit j of s lands on bit inv[j]
        for (int c = 0; c < T.nchunk; ++c)
            for (int val = 0; val < 256; ++val) {
                uint64_t r = 0;
                for (int k = 0; k < 8; ++k) {
                    const int j = 8 * c + k;
                    if (j < N && ((val >> k) & 1)) r |= 1ull << inv[j];
                }
                T.act[((size_t)g * T.nchunk + c) * 256 + val] = r;
            }
    }
    std::unordered_map<std::string, int> index;  // permutation -> group index
    auto key = [&](const int32_t *q) { return std::string((const char *)q, sizeof(int32_t) * N); };
    for (int g = 0; g < G; ++g) index.emplace(key(perm(g)), g);
    for (int Lx = 2; Lx <= 8 && !T.tx; ++Lx) {
        if (N % Lx || G % N) continue;
        const int Ly = N / Lx, nt = N;
        std::vector<int32_t> q(N);
        std::vector<int> tr(nt, -1);  // group index of T_{a,b}, at a + Lx b
        bool ok = true;
        for (int t = 0; t < nt && ok; ++t) {
            const int a = t % Lx, bb = t / Lx;
            for (int i = 0; i < N; ++i) q[i] = ((i % Lx + a) % Lx) + Lx * ((i / Lx + bb) % Ly);
            auto it = index.find(key(q.data()));
            if (it == index.end()) ok = false;
            else tr[t] = it->second;
        }
        if (!ok) continue;
        // the identity (tr[0]) first, so that p_0 is the identity
        std::vector<int16_t> tg, tpp;
        std::vector<char> covered(G, 0);
        for (int n = -1; n < G && ok; ++n) {
            const int g = n < 0 ? tr[0] : n;
            if (covered[g]) continue;
            tpp.push_back((int16_t)g);
            for (int t = 0; t < nt && ok; ++t) {
                const int32_t *pt = perm(tr[t]);
                for (int i = 0; i < N; ++i) q[i] = perm(g)[pt[i]];
                auto it = index.find(key(q.data()));
                if (it == index.end() || covered[it->second]) {
                    ok = false;
                } else {
                    covered[it->second] = 1;
                    tg.push_back((int16_t)it->second);
                }
            }
        }
        if (!ok || (int)tpp.size() * nt != G) continue;
        T.minrot.assign(1u << Lx, 0);
        T.amask.assign(1u << Lx, 0);
        for (uint32_t r = 0; r < (1u << Lx); ++r) {
            uint32_t m = r, mask = 0;
            for (int a = 0; a < Lx; ++a) {
                const uint32_t rr = ((r >> a) | (r << (Lx - a))) & ((1u << Lx) - 1);
                if (rr < m) {
                    m = rr;
                    mask = 1u << a;
                } else if (rr == m) {
                    mask |= 1u << a;
                }
            }
            T.minrot[r] = (uint8_t)m;
            T.amask[r] = (uint8_t)mask;
        }
        if (Lx <= 7) {
            T.cut.assign((size_t)1 << (2 * Lx), 0);
            for (uint32_t r = 0; r < (1u << Lx); ++r)
                for (uint32_t A = 1; A < (1u << Lx); ++A) {
                    uint32_t m = 0xffu, sub = 0;
                    for (int a = 0; a < Lx; ++a) {
                        if (!((A >> a) & 1)) continue;
                        const uint32_t rr = ((r >> a) | (r << (Lx - a))) & ((1u << Lx) - 1);
                        if (rr < m) {
                            m = rr;
                            sub = 1u << a;
                        } else if (rr == m) {
                            sub |= 1u << a;
                        }
                    }
                    T.cut[((size_t)r << Lx) | A] = (uint16_t)(m | (sub << 8));
                }
        }
        T.tx = Lx;
        T.ty = Ly;
        T.tnp = tpp.size() > 1 ? (int)tpp.size() : 0;
        T.tg = tg;
        T.tpp = tpp;
        T.pm.assign((size_t)(T.tnp > 1 ? T.tnp - 1 : 0) * nb, 0);
        for (int k = 1; k < T.tnp; ++k) {
            for (int i = 0; i < N; ++i) inv[perm(tpp[k])[i]] = i;
            for (int b = 0; b < nb; ++b)
                T.pm[(size_t)(k - 1) * nb + b] = (1ull << inv[bonds[2 * b]]) | (1ull << inv[bonds[2 * b + 1]]);
        }
    }
    if (!T.tx && N <= 64 && (G == N || G == 2 * N)) {
        std::vector<int16_t> cg(2 * N, -1);
        bool ok = true;
        for (int g = 0; g < G && ok; ++g) {
            const int32_t *p = perm(g);
            const int n = p[0];
            bool rot = true, ref = true;
            for (int i = 0; i < N; ++i) {
                rot = rot && p[i] == (i + n) % N;
                ref = ref && p[i] == ((n - i) % N + N) % N;
            }
            if (N > 2 && rot && ref) ok = false;  // only the identity of N <= 2 is both
            const int slot = rot ? n : ref ? N + n : -1;
            if (slot < 0 || cg[slot] >= 0) ok = false;
            else cg[slot] = (int16_t)g;
        }
        int nrot = 0, nref = 0;
        for (int n = 0; n < N; ++n) {
            nrot += cg[n] >= 0;
            nref += cg[N + n] >= 0;
        }
        if (ok && nrot == N && (nref == 0 || nref == N) && N + nref == G) {
            T.cn = N;
            T.cdih = nref ? 1 : 0;
            T.cg = cg;
        }
    }
}

}  // namespace xd
