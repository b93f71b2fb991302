// Reverse-mode launchers, float.
#include "adj_impl.cuh"

MPA_ADJ_INSTANTIATE(float)
