// Host check of the flat split's tables (test program; no GPU work). For each (L, G) given
// on the command line, builds the tables with flat_split_tables and walks them the way the
// history-integral kernels do (warp g takes the pairs of its segment row by row; each piece
// is part g - row[j].x of row[j].y), then checks:
//   - the segment starts are non-decreasing, segment g starts at pair g L^2 / G, and every
//     segment is non-empty (flat_split_fits holds for every case given);
//   - every row's pieces arrive in part order 0, 1, ..., nparts - 1, are contiguous and
//     cover the row's L pairs exactly once, so every pair is summed once;
//   - a row has at most max(L / 32, 1) parts (the partial-sum buffer's capacity).
// Prints "ok <cases>" or the first failure.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2604_06309_gb300/csrc/hi_units.h"

static int check(int L, int G) {
    std::vector<int2> seg, row;
    flat_split_tables(L, G, seg, row);
    const long long LL = (long long)L * L;
    if ((int)seg.size() != G + 1 || (int)row.size() != L) return 1;
    if (seg[0].x != 0 || seg[0].y != 0 || seg[G].x != LL || seg[G].y != L) return 2;
    for (int g = 0; g < G; ++g) {
        if (seg[g].x != (long long)g * LL / G) return 3;
        if (seg[g + 1].x <= seg[g].x) return 4;
        if (seg[g].y != seg[g].x / L) return 5;
    }
    std::vector<int> next_part(L, 0), end_i(L, 0);
    for (int g = 0; g < G; ++g) {
        const int2 a = seg[g], b = seg[g + 1];
        int j = a.y;
        for (int q = a.x; q < b.x; ++j) {
            if (j >= L) return 6;
            const int rb = j * L;
            const int qe = b.x < rb + L ? b.x : rb + L;
            const int2 r = row[j];
            const int part = g - r.x, nparts = r.y;
            if (part < 0 || part >= nparts) return 7;
            if (part != next_part[j]) return 8;
            if (q - rb != end_i[j]) return 9;
            next_part[j] += 1;
            end_i[j] = qe - rb;
            q = qe;
        }
    }
    const int cap = L / 32 > 1 ? L / 32 : 1;
    for (int j = 0; j < L; ++j) {
        if (end_i[j] != L) return 10;
        if (next_part[j] != row[j].y) return 11;
        if (row[j].y > cap) return 12;
    }
    return 0;
}

int main(int argc, char** argv) {
    int cases = 0;
    for (int k = 1; k + 1 < argc; k += 2) {
        const int L = std::atoi(argv[k]), G = std::atoi(argv[k + 1]);
        if (!flat_split_fits(L, G)) {
            std::printf("case L=%d G=%d does not fit\n", L, G);
            return 1;
        }
        const int rc = check(L, G);
        if (rc) {
            std::printf("fail L=%d G=%d check %d\n", L, G, rc);
            return 1;
        }
        ++cases;
    }
    std::printf("ok %d\n", cases);
    return 0;
}
