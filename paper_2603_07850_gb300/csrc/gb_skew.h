// gb_skew.h -- host-side table of the tier-A lane skews (plain C++, no CUDA;
// the library builds it once per process, the CPU tests check it).
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <algorithm>

namespace gbk {

// Lane skews of the tier-A marks.  In a warp-per-prime pass lane l marks the
// multiples l, l + 32, ... of p: one warp step touches the words
// floor((r + l p) / 32) + const, r = the first bit mod 32, and their
// shared-memory banks (word mod 32) collide for many p.  Lane l may start at
// its d_l-th multiple (d_l < 4) and mark its first d_l last, which moves its
// bank by d_l p.  For each (p mod 1024, r) -- all the banks depend on -- the
// d_l come from a bipartite matching of lanes to banks in which every bank
// takes at most c lanes, c as small as possible, smaller d_l tried first
// (augmenting paths, Kuhn 1955).  Entry ((p mod 1024) >> 1) * 32 + r holds d_l
// in bits 2l, 2l + 1.  The marks are the same in any order.
constexpr size_t ASKEW_ENTRIES = 512 * 32;

struct SkewMatch {
    int opt[32][4];
    int cap;
    int lanes[32][32], nl[32];               // lanes assigned to each bank
    int choice[32];
    bool seen[32];
    bool aug(int l)
    {
        for (int d = 0; d < 4; d++) {
            const int b = opt[l][d];
            if (seen[b]) continue;
            seen[b] = true;
            if (nl[b] < cap) {
                lanes[b][nl[b]++] = l;
                choice[l] = d;
                return true;
            }
            for (int i = 0; i < nl[b]; i++) {
                if (aug(lanes[b][i])) {              // that lane moved to another bank
                    lanes[b][i] = l;
                    choice[l] = d;
                    return true;
                }
            }
        }
        return false;
    }
};

// Fill tab[0 .. ASKEW_ENTRIES) with the skews.
inline void tier_a_skew_table(unsigned long long *tab)
{
    for (uint32_t h = 0; h < 512; h++) {
        const uint32_t p = 2 * h + 1;                // p mod 1024: the banks depend on nothing else
        for (uint32_t r = 0; r < 32; r++) {
            SkewMatch m;
            for (int l = 0; l < 32; l++)
                for (int d = 0; d < 4; d++) m.opt[l][d] = (int)((((r + (uint32_t)l * p) >> 5) + (uint32_t)d * p) & 31u);
            for (m.cap = 1; m.cap <= 32; m.cap++) {
                std::fill(m.nl, m.nl + 32, 0);
                bool ok = true;
                for (int l = 0; l < 32 && ok; l++) {
                    std::fill(m.seen, m.seen + 32, false);
                    ok = m.aug(l);
                }
                if (ok) break;
            }
            unsigned long long e = 0;
            for (int l = 0; l < 32; l++) e |= (unsigned long long)m.choice[l] << (2 * l);
            tab[h * 32 + r] = e;
        }
    }
}

}  // namespace gbk
