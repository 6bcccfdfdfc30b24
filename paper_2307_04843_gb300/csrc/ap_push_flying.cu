// ap_push_flying.cu -- kernels and launchers of the gather + push for pulse kind AP_FLYING_SUM.
#include "ap_kernels.cuh"

APT_DEFINE_KIND(flying, AP_FLYING_SUM)
