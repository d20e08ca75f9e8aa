// code.h -- the library-owned result of an encode (opaque aqmp_code of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "../../include/aqmp.h"
#include "common.cuh"

struct aqmp_code {
    int device = 0;
    int dict_id = 0, min_block = 4, max_block = 64;
    std::vector<std::pair<int, int>> shapes;      // (h, w) per plane
    aqmp::LeafRec *leaves = nullptr;              // device, canonical order
    aqmp::AtomRec *atoms = nullptr;               // device
    float *alpha_lo = nullptr;                    // device
    unsigned long long n_leaves = 0, n_atoms = 0;
    aqmp_stats stats{};
    ~aqmp_code() {
        if (leaves) cudaFree(leaves);
        if (atoms) cudaFree(atoms);
        if (alpha_lo) cudaFree(alpha_lo);
    }
};
