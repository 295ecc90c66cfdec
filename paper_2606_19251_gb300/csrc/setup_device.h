// AMG setup on the device (Sec. 2.2 with a parallel C/F split): strength
// graph, block-local RS or PMIS splitting, direct interpolation, R = P^T and the Galerkin
// product A_c = R (A P), every level built by CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "setup_host.h"

namespace amg {

// Setup-AMG-Hierarchy of Algorithm 1 on the device.  split_mode is a set of
// AMG_SPLIT_* flags: AMG_SPLIT_RS_BLOCKS takes the block-local RS first pass
// (with the repair of F points left without a strong C point) instead of
// PMIS; AMG_SPLIT_SECOND_PASS adds the round-parallel second pass (every
// strong F-F pair gets a common strong C point).  Level l draws its random
// numbers r_i = top 53 bits of splitmix64(seed + l) output i + 1, times
// 2^-53.  Same stopping rules as the host RS setup.  Returns AMG_OK or
// AMG_ERR_CUDA (message in err).
//
// The levels stay on the device: every HostCSR of `levels` holds its row
// pointers on the host and its columns and values only as device pointers
// (drp, dcol, dval) into memory that `keep` owns; the caller copies them
// where it needs them and then releases `keep`.
int device_build_hierarchy(const HostCSR &A0, double theta, int max_levels, int max_coarse,
                           unsigned long long seed, int split_mode, cudaStream_t s,
                           std::vector<HostLevel> &levels, std::shared_ptr<void> &keep, std::string &err);

// For every level l with which[l] set (R and A present), computed on the
// device and stored into levels[l]: MA = the pattern of A A (columns sorted,
// values zero; the pattern of M A for M = Q^-1 on A's pattern), the pair list
// that assembles its values, (M A)[e] = sum over t in
// [pair_ptr[e], pair_ptr[e+1]) of M[pair_p[t]] * A[pair_q[t]] with each
// entry's pairs in ascending p, and RA = R A.  Returns AMG_OK or AMG_ERR_CUDA
// (message in err).
int device_plan_products(std::vector<HostLevel> &levels, const std::vector<char> &which, cudaStream_t s,
                         std::string &err);

}  // namespace amg
