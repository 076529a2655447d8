// Team sizes of the Newton wavefront: host code shared by pit_create (one problem) and the
// batched solver's wavefront jobs. Plain C++, no CUDA.
#pragma once

#include <algorithm>
#include <cstdlib>

// K teams (Newton iterations in flight) of Gw CTAs share ny grid rows of nx nodes as row strips
// on P SMs. The SMs that the K equal teams leave over go to the teams nearest the middle:
//   - order: |2t - K| ascending, lower t first on ties;
//   - each upgraded team takes the fewest CTAs whose strips are shorter (at most rows - 1 rows);
//   - only within the automatic team size's cap (a CTA per min_local unknowns: ceil(ny / rows_min)
//     CTAs, rows_min = ceil(min_local / nx)) and at most max_team CTAs.
// Under the forcing terms the middle Newton iterations take the most sweeps per level (burgers256,
// FP64: 5.6, 6.0, 7.5, 8.2, 5.7 and 1.3 for iterations 0-5). The slowest iteration's level chain
// paces the ones after it, so a shorter strip there shortens the launch.
// fixed > 0 keeps every team at Gw. sizes[0..K) receives the teams' CTA counts; returns their sum.
inline int pit_wave_team_sizes(int K, int Gw, int nx, int ny, int P, int min_local, int max_team, int fixed,
                               int* sizes) {
    for (int t = 0; t < K; ++t) sizes[t] = Gw;
    const int rows = (ny + Gw - 1) / Gw;
    const int rows_min = (min_local + nx - 1) / nx;
    int G2 = rows > 2 ? (ny + rows - 2) / (rows - 1) : Gw;  // the fewest CTAs whose strips are shorter
    if (G2 > (ny + rows_min - 1) / rows_min) G2 = Gw;        // the automatic size's cap
    if (K >= 2 && fixed <= 0 && G2 > Gw && G2 <= max_team && P > K * Gw) {
        const int n_up = std::min(K, (P - K * Gw) / (G2 - Gw));
        int order[64];
        const int n = std::min(K, 64);
        for (int t = 0; t < n; ++t) order[t] = t;
        std::stable_sort(order, order + n, [K](int x, int y) { return std::abs(2 * x - K) < std::abs(2 * y - K); });
        for (int i = 0; i < std::min(n_up, n); ++i) sizes[order[i]] = G2;
    }
    int total = 0;
    for (int t = 0; t < K; ++t) total += sizes[t];
    return total;
}
