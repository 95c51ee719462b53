"""GB300-native IonTracks charge-carrier transport step (arXiv:1610.06749)."""
