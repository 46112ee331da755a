// densify.cuh -- one Delaunay densification step (Sec. 4, Alg. 1).
#pragma once
int Ctx::densify(const hdi_image*, hdi_mask*, const hdi_image*, int64_t, uint64_t, int64_t*) {
    return fail(HDI_ERR_UNSUPPORTED, "densification not built yet");
}
