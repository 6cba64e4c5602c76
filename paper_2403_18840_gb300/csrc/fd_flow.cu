// Affine coupling flow: entry points (kernels follow in this file).
#include "fd_internal.cuh"

extern "C" fd_status fd_flow_create(int32_t, int32_t, int32_t, uint64_t, fd_flow **out) {
    if (out) *out = nullptr;
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
extern "C" void fd_flow_free(fd_flow *) {}
extern "C" int64_t fd_flow_param_count(const fd_flow *) { return 0; }
extern "C" fd_status fd_flow_set_params(fd_flow *, const float *, int64_t) {
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
extern "C" fd_status fd_flow_get_params(const fd_flow *, float *, int64_t) {
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
extern "C" fd_status fd_flow_sample(const fd_flow *, uint64_t, uint64_t, int32_t, int64_t, float *, float *, void *) {
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
extern "C" fd_status fd_flow_log_density(const fd_flow *, const float *, int64_t, float *, void *) {
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
extern "C" fd_status fd_flow_grad(fd_flow *, const float *, const float *, int64_t, float *, float *, void *) {
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
extern "C" fd_status fd_flow_train(fd_flow *, const float *, const float *, int64_t, int32_t, float, float *, void *) {
    return fd::set_error(FD_ENOTSUP, "flow kernels not built yet");
}
