// Declarations of the randomised copies (double-edge swaps on the device).
#pragma once

#include "common.cuh"

namespace acc {

// randomise.cu: randomised copies of a set of graphs.  Graph g's copies
// start at element ooff of the output, copy r at ooff + r * m, and use the
// SplitMix64 stream seeded seed + r.
struct RGraph {
    const long long *rowptr;  // input out-CSR (device)
    const int *col;
    long long m;
    long long moff;           // first arc of the graph in the set's numbering (row table)
    long long ooff;           // first element of the graph's copies in the output
    long long attempts;       // swap attempts per copy
    unsigned long long seed;  // stream of copy 0
    long long boff;           // first word of the graph's copies' adjacency bitmaps
    int n;
    int voff;                 // first vertex of the graph in the set's numbering
    int bw;                   // bitmap words per row (a multiple of 4)
    int pad;
};
// Validates the graphs and fills rows (int4[M]: begin, end, source of each
// position), then runs the copies (mode ACC_RAND_SWAP or ACC_RAND_MUTUAL);
// the copies are skipped when *status is set.  With bits non-null (R times
// the graphs' n * bw words) the plain mode runs the speculative kernel, and
// so does the mutual mode when rpart (M ints: reverse position of each arc)
// and pts (R * M ints: the copies' reverse positions) are non-null too.
int launch_randomise(const RGraph *meta, int G, int R, long long M, long long NV, int mode, int4 *rows, int *out,
                     uint32_t *bits, int *rpart, int *pts, long long *accepted, int *status, int num_sms,
                     cudaStream_t s);

}  // namespace acc
