// Entry points whose kernels are not in this build yet: they validate nothing
// and return PANTHER_EINVAL with a message, so the ABI is complete.
#include "internal.cuh"

extern "C" {
panther_status panther_serve_create(int, const panther_index*, const panther_paths*, const pantherpp_vecs*, int64_t,
                                    int, int, panther_server** out) {
    if (out) *out = nullptr;
    return PANTHER_EINVAL;
}
panther_status panther_serve_submit(panther_server*, int, const int32_t*, int64_t, int, int32_t*, void*, int64_t*) {
    return PANTHER_EINVAL;
}
panther_status panther_serve_wait(panther_server*, int64_t, double, double*) { return PANTHER_EINVAL; }
panther_status panther_serve_stats(panther_server*, int64_t*) { return PANTHER_EINVAL; }
void panther_serve_destroy(panther_server*) {}
}
