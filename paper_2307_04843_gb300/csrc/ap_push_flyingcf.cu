// ap_push_flyingcf.cu -- kernels and launchers of the gather + push for pulse kind AP_FLYING_CF.
#include "ap_kernels.cuh"

APT_DEFINE_KIND(flyingcf, AP_FLYING_CF)
