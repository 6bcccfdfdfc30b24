// ap_push_gauss.cu -- kernels and launchers of the gather + push for pulse kind AP_GAUSS.
#include "ap_kernels.cuh"

APT_DEFINE_KIND(gauss, AP_GAUSS)
