// Worklist records shared by the apply kernels (apply.cu, apply_fact.cu).
#pragma once
#include "mra_internal.cuh"

namespace mra {

struct Pair {
    int32_t out;    // output node
    int32_t in;     // input node (>= 0) or -1 - ghost id
    int16_t m_lo, m_hi;
    int8_t t1, t2, t3;
    uint8_t flags;  // bit 0: core translation at an internal node
};
static_assert(sizeof(Pair) == 16, "Pair is 16 bytes");

struct ApplyArgs {
    int k, M, n;
    const Pair* pairs;
    const int32_t* pair_off;
    const int32_t* coord;
    const double* s;
    const double* gblk;
    const double* w;
    const void* F;         // double or float table [j][m][l+3][k][k]
    const double* nF;
    const int32_t* Jm;
    double eta_blk;        // < 0: no per-block screen
    double* out;
    unsigned long long* n_items;
};

int launch_apply_fact(const ApplyArgs& A, int precision, int nlev, cudaStream_t st);
int launch_apply_tc(const ApplyArgs& A, int nghost, int nlev, const mra_op* op, int* err, cudaStream_t st);

}  // namespace mra
