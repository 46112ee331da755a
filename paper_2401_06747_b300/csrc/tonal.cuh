// tonal.cuh -- RAS tonal optimisation (Sec. 5.2, Alg. 2).
#pragma once
int Ctx::tonal(const hdi_image*, const hdi_mask*, const hdi_image*, hdi_image*, double, hdi_stats*) {
    return fail(HDI_ERR_UNSUPPORTED, "tonal optimisation not built yet");
}
