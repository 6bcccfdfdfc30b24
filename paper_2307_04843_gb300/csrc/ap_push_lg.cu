// ap_push_lg.cu -- kernels and launchers of the gather + push for pulse kind AP_LG.
#include "ap_kernels.cuh"

APT_DEFINE_KIND(lg, AP_LG)
