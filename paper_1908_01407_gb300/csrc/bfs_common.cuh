// Argument and state blocks of the BFS kernels (shared with the
// multi-source BFS and the serving loop).
#pragma once
#include "common.cuh"

namespace gbx {

// What a launch reports; block 0 thread 0 writes it, the last block to
// leave the kernel adds the error code.
struct BfsResult {
    int err;
    unsigned int depth, push_levels, pull_levels;
    unsigned long long edges_examined;
    unsigned long long frontier_edges;
    unsigned long long reached;
    double alg_bytes;
    unsigned long long t_begin;        // %globaltimer after the initial grid barrier
    unsigned long long t_entry;        // block 0 entering the kernel
    unsigned long long t_end;          // block 0 leaving the level loop
    unsigned long long t_exit;         // the last block leaving the kernel
    unsigned int dir_log[GBX_MAX_LEVEL_LOG];        // 1 = push, 2 = pull
    unsigned int lv_cnt[GBX_MAX_LEVEL_LOG];         // frontier vertices per level
    unsigned long long lv_fe[GBX_MAX_LEVEL_LOG];    // frontier out-edges per level
    unsigned long long lv_ns[GBX_MAX_LEVEL_LOG];    // %globaltimer at each level start
};

static_assert(sizeof(BfsResult) % 8 == 0, "BfsResult is zeroed in 8-byte words");

// Working state. It is all zero when a launch starts: the last block to
// leave a launch zeroes it again (so no memset is needed between launches).
struct BfsState {
    dev::GridBarrier bar;
    int err;
    int pad0;
    unsigned long long qstate[3];      // packed (list length << ebits | edge-prefix total), per level slot
    unsigned long long exam[3];        // adjacency entries read by pull, per level slot
    unsigned long long cstate[3];      // packed counter of the bitmap -> list compaction, per level slot
    unsigned int ucnt[3];              // length of the candidate list a pull leaves, per pull slot
    unsigned int pad1;
    unsigned long long uedg[3];        // in-edges of the candidates a pull leaves, per pull slot
    unsigned long long uact[3];        // unvisited candidates a pull walked, per level slot
    unsigned int far_cnt;              // SSSP near-far: vertices in the far set
    int sticky;                        // max of the exit codes of launches nobody has waited for yet
                                       // (launches leave it as it is; gb_context_synchronize reads and clears it)
    BfsResult res;
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
    uint32_t *q[2], *qp[2], *qr[2];    // frontier list: vertex, out-edge prefix, row start
    const PullRec *live_rec;           // pull records of the vertices with an in-edge (ascending); null = none
    const uint32_t *live_count;        // device scalar: number of records
    void *ul[2];                       // candidate lists of the pull steps (unvisited, with in-edges): pull
                                       // records with the live table, vertex ids without it
    const uint32_t *comp_size;         // per vertex, its component's size; null = unknown
    int ebits;
    unsigned long long emask;
    int mode;
    uint32_t beta;
    BfsState *st;
    uint64_t timeout_ns;       // bound on one grid-barrier wait
    uint64_t total_limit_ns;   // bound on the whole traversal
    int *err_sticky;           // optional: a nonzero exit status is also max-ed in here (batched runs)
    int *status_out;           // optional: the exit status (0 or GB_TIMEOUT) is stored here by the last block
    bool withhold;             // failure-path test: block 0 never arrives at the first grid barrier
};

}  // namespace gbx
