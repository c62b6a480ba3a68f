"""GB300-native CDDT ray casting fused with the beam sensor model."""
