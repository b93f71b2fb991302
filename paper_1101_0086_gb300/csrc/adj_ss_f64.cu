// Reverse-mode launchers of the split-step, double.
#include "adj_impl.cuh"

MPA_ADJ_INSTANTIATE_SS(double)
