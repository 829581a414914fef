// Learned step-cost model (costmodel.cu) and the step features it reads.
#pragma once
#include <vector>

#include "tn.h"

namespace tn {

constexpr int kCostFeatures = 16;

// number of MLP parameters
int cost_params();

// log2(ms) predictions for a host feature matrix (rows of kCostFeatures);
// synchronous, on the legacy stream
int cost_predict_host(tn_costmodel_t cm, const std::vector<float> &X, std::vector<float> &Y);

}  // namespace tn
