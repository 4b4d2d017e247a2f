// xd_groups.h -- host-side questions about a bond list under a group of site
// permutations (Sec. 3.9-3.10): which bonds lie on one orbit, and whether the
// couplings are invariant.  Plain C++ without CUDA; bonds are [nb][2] site
// pairs, perms [G][N] with perms[g][i] = g(i).  A hash of the unordered site
// pair turns each question into G x nb lookups.
#pragma once

#include <stdint.h>

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

}  // namespace xd
