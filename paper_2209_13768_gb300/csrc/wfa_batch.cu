// Batched stepping of many grids (temporary sequential form; see wfa_step).
#include "wfa_internal.cuh"

extern "C" int wfa_batch_run(wfa_grid* gs, const long long* steps, int count) {
    if (count < 0 || (count > 0 && (!gs || !steps))) {
        wfa::set_error("wfa_batch_run: bad arguments");
        return WFA_ERR_ARG;
    }
    for (int i = 0; i < count; ++i) {
        int rc = wfa_step(gs[i], steps[i]);
        if (rc) return rc;
    }
    return WFA_OK;
}
