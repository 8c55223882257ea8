// Channel-averaging tables (Sec. 2.6), one definition for host and device code: the plan
// path builds them on the host, the allocation-free call builds them inside a set-up
// kernel.  Both get the same bits: only IEEE-exact operations (add, divide, square root).
#pragma once

#include "mwax_internal.cuh"

namespace mwax {

// Output channel j of M = keep/F is centred on ultrafine offset (j - floor(M/2)) F; odd F
// takes F bins of weight 1, even F takes F+1 bins with the two ends at 1/2; the DC bin is
// dropped from the centre channel when F > 1 (unless kept); bins beyond the kept band (the
// coarse channel, or its central keep bins when oversampled, Sec. 4.5) do not exist.
// Writes gain[c] = sqrt(w_c) for the N ultrafine channels and the groups of consecutive
// channels that feed the same output channels (coef = 1 / sum(w), first_a / first_b set
// on the first group feeding each output channel).  Returns the number of groups, or -1
// when the averaging is inconsistent: an output channel with no weight, a bin carrying two
// different weights, a bin feeding more than two output channels, or more groups than
// max_groups.  Caller-provided scratch: w[N], fa[N], fb[N], wsum[M], seen[M].
__host__ __device__ inline int build_avg_groups(int N, int keep, int F, int dc_excl, float* gain, Group* groups,
                                                int max_groups, double* w, int* fa, int* fb, double* wsum,
                                                char* seen)
{
    const int M = keep / F, jc = M / 2, half = F / 2;
    for (int c = 0; c < N; ++c) {
        w[c] = 0.0;
        fa[c] = fb[c] = -1;
    }
    for (int j = 0; j < M; ++j) {
        wsum[j] = 0.0;
        seen[j] = 0;
    }
    for (int j = 0; j < M; ++j) {
        const long long mid = (long long)(j - jc) * F;
        for (long long u = mid - half; u <= mid + half; ++u) {
            if (u < -(keep / 2) || u > keep - keep / 2 - 1) continue;   // outside the kept band
            const int c = (int)(u + N / 2);
            double wt = (F % 2 == 0 && (u == mid - half || u == mid + half)) ? 0.5 : 1.0;
            if (dc_excl && F > 1 && u == 0) wt = 0.0;
            if (wt == 0.0) continue;
            if (w[c] != 0.0 && w[c] != wt) return -1;   // a bin has one weight everywhere
            w[c] = wt;
            if (fa[c] < 0) fa[c] = j;
            else if (fb[c] < 0) fb[c] = j;
            else return -1;                              // at most two output channels per bin
            wsum[j] += wt;
        }
    }
    for (int j = 0; j < M; ++j)
        if (wsum[j] <= 0.0) return -1;
    int ng = 0;
    for (int c = 0; c < N; ++c) {
        gain[c] = (float)sqrt(w[c]);
        if (w[c] == 0.0) continue;
        if (ng > 0 && groups[ng - 1].ja == fa[c] && groups[ng - 1].jb == fb[c]) {
            groups[ng - 1].c1 = c + 1;   // zero-weight channels in between are skipped by the kernels
            continue;
        }
        if (ng == max_groups) return -1;
        Group& g = groups[ng++];
        g.c0 = c;
        g.c1 = c + 1;
        g.ja = fa[c];
        g.jb = fb[c];
        g.ca = (float)(1.0 / wsum[fa[c]]);
        g.cb = fb[c] >= 0 ? (float)(1.0 / wsum[fb[c]]) : 0.0f;
        // groups are in channel order and a run always starts at the first group of its
        // first channel, so the first group met for a channel is the one that stores
        g.first_a = !seen[g.ja];
        seen[g.ja] = 1;
        g.first_b = 0;
        if (g.jb >= 0) {
            g.first_b = !seen[g.jb];
            seen[g.jb] = 1;
        }
    }
    return ng;
}

}  // namespace mwax
