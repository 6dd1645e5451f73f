// batch.cu -- many grids per launch (placeholder until the work-list kernel lands).
#include "spfm_internal.h"

extern "C" {
spfm_status spfm_batch_scratch_bytes(spfm_grid *const *, int, size_t *bytes)
{
    if (bytes) *bytes = 0;
    return SPFM_EINVAL;
}
spfm_status spfm_batch_create(spfm_grid *const *, int, void *, size_t, void *, spfm_batch **out)
{
    if (out) *out = nullptr;
    return SPFM_EINVAL;
}
spfm_status spfm_batch_step(spfm_batch *, int, const spfm_step_args *) { return SPFM_EINVAL; }
spfm_status spfm_batch_stats(spfm_batch *, int, spfm_stats *) { return SPFM_EINVAL; }
spfm_status spfm_batch_destroy(spfm_batch *) { return SPFM_OK; }
}
