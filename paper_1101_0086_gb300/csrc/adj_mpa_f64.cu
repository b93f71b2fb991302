// Reverse-mode launchers of the MPA, double.
#include "adj_impl.cuh"

MPA_ADJ_INSTANTIATE_MPA(double)
