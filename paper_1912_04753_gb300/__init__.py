"""GB300-native space-time Ripley's K (edge-corrected K / L and CSR simulation envelopes)."""
