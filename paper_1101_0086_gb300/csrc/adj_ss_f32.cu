// Reverse-mode launchers of the split-step, float.
#include "adj_impl.cuh"

MPA_ADJ_INSTANTIATE_SS(float)
