// ap_push_plane.cu -- kernels and launchers of the gather + push for pulse kind AP_PLANE.
#include "ap_kernels.cuh"

APT_DEFINE_KIND(plane, AP_PLANE)
