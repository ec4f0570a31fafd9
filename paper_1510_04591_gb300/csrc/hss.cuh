// HSS update path (Algorithms 2 and 3, SRRSC) -- internal interface.
#pragma once

#include <string>
#include <vector>

#include "../../include/tdeig.h"
#include "common.cuh"

struct HssWS {
    double* pool;      // generator / sampling storage
    size_t pool_elems;
    int* ipool;
    size_t ipool_elems;
};

struct Arena;
size_t hss_ws_bytes(const tdeig_options& opt, int64_t Qsz, int64_t R, bool enabled);
void hss_carve_ws(Arena& a, HssWS& w, const tdeig_options& opt, int64_t Qsz, int64_t R, bool enabled);
int hss_update_level(const tdeig_options& opt, int variant, int prec,
                     const std::vector<MergeDesc>& merges, const MergeDesc* dev_merges,
                     const std::vector<int>& K, const LevelWS& lws, HssWS& hws, int* status,
                     cudaStream_t st, std::string& stats);
