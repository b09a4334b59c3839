"""B300-native neural receiver (NRX) forward pass and LS+LMMSE receiver."""
