// Argument and state blocks of the BFS kernels (shared with the
// multi-source BFS and the serving loop).
#pragma once
#include "common.cuh"

namespace gbx {

struct BfsState {
    dev::GridBarrier bar;
    int err;
    int pad0;
    unsigned long long qstate[3];      // packed (list length << ebits | edge-prefix total), per level slot
    unsigned long long exam[3];        // adjacency entries read by pull, per level slot
    unsigned long long edges_examined;
    unsigned long long frontier_edges;
    unsigned long long reached;
    double alg_bytes;
    unsigned int depth, push_levels, pull_levels, pad1;
    unsigned int dir_log[GBX_MAX_LEVEL_LOG];   // 1 = push, 2 = pull
};

struct BfsArgs {
    const uint32_t *rp_out, *ci_out;   // CSR: out-neighbours (push)
    const uint32_t *rp_in, *ci_in;     // CSC: in-neighbours (pull); null = push only
    bool csr_is_csc;
    uint32_t n, nwords;
    uint64_t m;
    uint32_t src;
    int32_t *levels, *parents;
    uint32_t *visited;
    uint32_t *front[3];
    uint32_t *q[2], *qp[2];
    int ebits;
    unsigned long long emask;
    int mode;
    uint32_t beta;
    BfsState *st;
    uint64_t timeout_ns;       // bound on one grid-barrier wait
    uint64_t total_limit_ns;   // bound on the whole traversal
    uint64_t t_start_hint;     // 0: each block reads the clock itself
};

}  // namespace gbx
