// HSS construction (Algorithm 2, SRRSC) and HSS-times-matrix (Algorithm 3).
#include "hss.cuh"

size_t hss_ws_bytes(const tdeig_options&, int64_t, int64_t, bool) { return 0; }
void hss_carve_ws(Arena&, HssWS& w, const tdeig_options&, int64_t, int64_t, bool)
{
    w.pool = nullptr; w.pool_elems = 0; w.ipool = nullptr; w.ipool_elems = 0;
}
int hss_update_level(const tdeig_options&, int, int, const std::vector<MergeDesc>&,
                     const MergeDesc*, const std::vector<int>&, const LevelWS&, HssWS&, int*,
                     cudaStream_t, std::string&)
{
    return TDEIG_ENOTIMPL;
}
