// Reverse-mode launchers of the MPA, float.
#include "adj_impl.cuh"

MPA_ADJ_INSTANTIATE_MPA(float)
